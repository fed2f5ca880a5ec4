// Kernel instantiations: 3-DOF Mars descent, FP64 plain path.
#include "ucn_launch.cuh"
UCN_DEFINE_LAUNCHERS(mars64, Mars7, double, false)
