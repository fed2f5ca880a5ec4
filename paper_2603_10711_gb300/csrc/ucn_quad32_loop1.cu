// Device-resident request loop of a server: 12-state quadrotor, FP32 path with refinement; one thread
// per node, node records in shared memory.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Quad12, float, true, true, 1)
