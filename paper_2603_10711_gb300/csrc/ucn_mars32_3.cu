// Kernel instantiation: 3-DOF Mars descent, FP32 path with refinement, the
// one-thread fused solve in its three-CTAs-per-SM register class (records in
// shared memory).
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCP3(Mars7, float, true, true)
