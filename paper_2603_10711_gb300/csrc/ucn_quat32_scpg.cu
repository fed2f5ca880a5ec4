// Kernel instantiation: 13-state quaternion quadrotor, FP32 path with refinement, fused solve with
// node records in global memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP(Quat13, float, false, true)
