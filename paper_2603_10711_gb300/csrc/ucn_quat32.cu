// Kernel instantiations: 13-state quaternion quadrotor, FP32 path with refinement.  The fused
// solve with global-memory records and the stand-alone ADMM compile in their
// own units (ucn_quat32_*.cu).
#include "ucn_launch.cuh"
UCN_EXTERN_SCP(Quat13, float, false, true)
UCN_EXTERN_ADMM(Quat13, float, true, true)
UCN_EXTERN_ADMM(Quat13, float, false, true)
UCN_DEFINE_LAUNCHERS(quat32, Quat13, float, true)
