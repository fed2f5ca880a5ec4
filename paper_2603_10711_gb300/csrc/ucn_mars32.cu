// Kernel instantiations: 3-DOF Mars descent, FP32 path with refinement (the pair
// kernel compiles in ucn_mars32_pair.cu).
#include "ucn_launch.cuh"
UCN_EXTERN_SCPP(Mars7, true)
UCN_DEFINE_LAUNCHERS(mars32, Mars7, float, true)
