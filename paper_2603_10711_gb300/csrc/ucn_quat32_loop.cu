// Device-resident request loop of a server: 13-state quaternion quadrotor, FP32 path with refinement;
// one thread per node, node records in shared memory here, the other variant in its own unit (compiled
// in parallel).
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_EXTERN_LOOP(Quat13, float, false, true, 1)
UCN_INSTANTIATE_LOOP(Quat13, float, true, true, 1)
UCN_DEFINE_LOOP_LAUNCHER(quat32, Quat13, float, true)
