// Kernel instantiations: 3-DOF Mars descent, FP32 path with refinement (the pair
// kernel compiles in ucn_mars32_pair.cu, the three-CTAs-per-SM variant in
// ucn_mars32_3.cu).
#include "ucn_launch.cuh"
UCN_EXTERN_SCPP(Mars7, true)
UCN_EXTERN_SCP3(Mars7, float, true, true)
UCN_DEFINE_LAUNCHERS(mars32, Mars7, float, true)
