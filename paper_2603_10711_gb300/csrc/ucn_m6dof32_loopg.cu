// Device-resident request loop of a server: 6-DOF Mars lander, FP32 path with refinement; one thread
// per node, node records in the global workspace.
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_INSTANTIATE_LOOP(Mars14, float, false, true, 1)
