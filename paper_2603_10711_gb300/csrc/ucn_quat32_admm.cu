// Kernel instantiations: 13-state quaternion quadrotor, FP32 path with refinement, stand-alone ADMM.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_ADMM(Quat13, float, true, true)
UCN_INSTANTIATE_ADMM(Quat13, float, false, true)
