// Kernel instantiation: 12-state quadrotor, FP64 plain path, fused solve with node
// records in global memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP(Quad12, double, false, false)
