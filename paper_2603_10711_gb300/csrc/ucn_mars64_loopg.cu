// Device-resident request loop of a server: 3-DOF Mars descent, FP64 plain path; one thread per node,
// node records in the global workspace.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Mars7, double, false, false, 1)
