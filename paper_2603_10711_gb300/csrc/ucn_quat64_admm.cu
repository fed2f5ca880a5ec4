// Kernel instantiations: 13-state quaternion quadrotor, FP64 plain path, stand-alone ADMM.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_ADMM(Quat13, double, true, false)
UCN_INSTANTIATE_ADMM(Quat13, double, false, false)
