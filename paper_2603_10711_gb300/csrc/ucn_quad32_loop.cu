// Device-resident request loop of a server: 12-state quadrotor, FP32 path with refinement; the lane
// layout (4 threads per node), node records in shared memory here, the other variants in their own
// units (compiled in parallel).
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_EXTERN_LOOP(Quad12, float, false, true, 4)
UCN_EXTERN_LOOP(Quad12, float, true, true, 1)
UCN_EXTERN_LOOP(Quad12, float, false, true, 1)
UCN_INSTANTIATE_LOOP(Quad12, float, true, true, 4)
UCN_DEFINE_LOOP_LAUNCHER(quad32, Quad12, float, true)
