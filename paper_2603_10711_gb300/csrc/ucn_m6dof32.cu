// Kernel instantiations: 14-state 6-DOF Mars landing, FP32 path with refinement.  The fused solve
// with global-memory records and the stand-alone ADMM compile in their own
// units (ucn_m6dof32_*.cu).
#include "ucn_launch.cuh"
UCN_EXTERN_SCP(Mars14, float, false, true)
UCN_EXTERN_ADMM(Mars14, float, true, true)
UCN_EXTERN_ADMM(Mars14, float, false, true)
UCN_DEFINE_LAUNCHERS(m6dof32, Mars14, float, true)
