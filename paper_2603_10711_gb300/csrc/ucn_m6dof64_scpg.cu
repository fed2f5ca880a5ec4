// Kernel instantiation: 14-state 6-DOF Mars landing, FP64 plain path, fused solve with
// node records in global memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP(Mars14, double, false, false)
