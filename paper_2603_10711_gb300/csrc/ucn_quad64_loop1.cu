// Device-resident request loop of a server: 12-state quadrotor, FP64 plain path; one thread per node,
// node records in shared memory.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Quad12, double, true, false, 1)
