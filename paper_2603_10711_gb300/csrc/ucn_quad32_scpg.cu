// Kernel instantiation: 12-state quadrotor, FP32 path with refinement, fused solve with node
// records in global memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP(Quad12, float, false, true)
