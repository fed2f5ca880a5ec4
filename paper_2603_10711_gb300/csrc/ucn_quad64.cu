// Kernel instantiations: 12-state quadrotor, FP64 plain path.  The slow-to-compile
// variants live in their own units (ucn_quad64_*.cu) and compile in parallel.
#include "ucn_launch.cuh"
UCN_EXTERN_SCP(Quad12, double, false, false)
UCN_EXTERN_SCPL(Quad12, double, true, false, ucn::LANES_MAX_THREADS)
UCN_EXTERN_SCPL(Quad12, double, true, false, ucn::LANES_WIDE_THREADS)
UCN_EXTERN_SCPL(Quad12, double, false, false, ucn::LANES_MAX_THREADS)
UCN_EXTERN_SCPL(Quad12, double, false, false, ucn::LANES_WIDE_THREADS)
UCN_EXTERN_ADMM(Quad12, double, true, false)
UCN_EXTERN_ADMM(Quad12, double, false, false)
UCN_DEFINE_LAUNCHERS(quad64, Quad12, double, false)
