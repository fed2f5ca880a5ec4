// Kernel instantiations: 13-state quaternion quadrotor, FP64 plain path.  The fused
// solve with global-memory records and the stand-alone ADMM compile in their
// own units (ucn_quat64_*.cu).
#include "ucn_launch.cuh"
UCN_EXTERN_SCP(Quat13, double, false, false)
UCN_EXTERN_ADMM(Quat13, double, true, false)
UCN_EXTERN_ADMM(Quat13, double, false, false)
UCN_DEFINE_LAUNCHERS(quat64, Quat13, double, false)
