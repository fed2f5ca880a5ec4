// Device-resident request loop of a server: 13-state quaternion quadrotor, FP32 path with refinement;
// one thread per node, node records in the global workspace.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Quat13, float, false, true, 1)
