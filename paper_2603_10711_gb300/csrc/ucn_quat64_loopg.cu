// Device-resident request loop of a server: 13-state quaternion quadrotor, FP64 plain path; one thread
// per node, node records in the global workspace.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Quat13, double, false, false, 1)
