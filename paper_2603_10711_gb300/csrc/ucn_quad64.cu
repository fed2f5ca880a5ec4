// Kernel instantiations: 12-state quadrotor, FP64 plain path.
#include "ucn_launch.cuh"
UCN_DEFINE_LAUNCHERS(quad64, Quad12, double, false)
