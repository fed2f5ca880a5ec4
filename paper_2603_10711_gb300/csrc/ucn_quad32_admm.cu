// Kernel instantiations: 12-state quadrotor, FP32 path with refinement, stand-alone ADMM.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_ADMM(Quad12, float, true, true)
UCN_INSTANTIATE_ADMM(Quad12, float, false, true)
