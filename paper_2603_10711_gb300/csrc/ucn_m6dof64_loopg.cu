// Device-resident request loop of a server: 6-DOF Mars lander, FP64 plain path; one thread per node,
// node records in the global workspace.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Mars14, double, false, false, 1)
