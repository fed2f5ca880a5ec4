// Kernel instantiations: 3-DOF Mars descent, FP32 path with refinement.
#include "ucn_launch.cuh"
UCN_DEFINE_LAUNCHERS(mars32, Mars7, float, true)
