// Kernel instantiations: 12-state quadrotor, FP64 plain path, stand-alone ADMM.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_ADMM(Quad12, double, true, false)
UCN_INSTANTIATE_ADMM(Quad12, double, false, false)
