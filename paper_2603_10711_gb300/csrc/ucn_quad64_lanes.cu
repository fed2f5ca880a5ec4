// Kernel instantiation: 12-state quadrotor, FP64 plain path, fused solve on the lane
// layout (4 threads per node) with node records in shared memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCPL(Quad12, double, true, false)
