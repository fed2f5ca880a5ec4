// Kernel instantiations: 14-state 6-DOF Mars landing, FP32 path with refinement, stand-alone ADMM.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_ADMM(Mars14, float, true, true)
UCN_INSTANTIATE_ADMM(Mars14, float, false, true)
