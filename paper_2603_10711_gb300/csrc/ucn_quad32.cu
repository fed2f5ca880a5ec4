// Kernel instantiations: 12-state quadrotor, FP32 path with refinement.
#include "ucn_launch.cuh"
UCN_DEFINE_LAUNCHERS(quad32, Quad12, float, true)
