// Kernel instantiations: 14-state 6-DOF Mars landing, FP64 plain path, stand-alone ADMM.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_ADMM(Mars14, double, true, false)
UCN_INSTANTIATE_ADMM(Mars14, double, false, false)
