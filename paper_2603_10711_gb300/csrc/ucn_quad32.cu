// Kernel instantiations: 12-state quadrotor, FP32 path with refinement.  The slow-to-compile
// variants live in their own units (ucn_quad32_*.cu) and compile in parallel.
#include "ucn_launch.cuh"
UCN_EXTERN_SCP(Quad12, float, false, true)
UCN_EXTERN_SCPL(Quad12, float, true, true, ucn::LANES_MAX_THREADS)
UCN_EXTERN_SCPL(Quad12, float, true, true, ucn::LANES_WIDE_THREADS)
UCN_EXTERN_SCPL(Quad12, float, false, true, ucn::LANES_MAX_THREADS)
UCN_EXTERN_SCPL(Quad12, float, false, true, ucn::LANES_WIDE_THREADS)
UCN_EXTERN_ADMM(Quad12, float, true, true)
UCN_EXTERN_ADMM(Quad12, float, false, true)
UCN_DEFINE_LAUNCHERS(quad32, Quad12, float, true)
