// Kernel instantiation: 14-state 6-DOF Mars landing, FP32 path with refinement, fused solve with
// node records in global memory.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP(Mars14, float, false, true)
