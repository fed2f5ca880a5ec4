// Kernel instantiation: 13-state quaternion quadrotor, FP64 plain path, fused solve with
// node records in global memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP(Quat13, double, false, false)
