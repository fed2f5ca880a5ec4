// Kernel instantiation: 3-DOF Mars descent, FP32 path with refinement, fused
// solve with two threads per node (node records in shared memory).
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCPP(Mars7, true)
