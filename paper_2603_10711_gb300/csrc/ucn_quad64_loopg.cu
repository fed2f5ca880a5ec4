// Device-resident request loop of a server: 12-state quadrotor, FP64 plain path; the lane layout (4
// threads per node), node records in the global workspace.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Quad12, double, false, false, 4)
