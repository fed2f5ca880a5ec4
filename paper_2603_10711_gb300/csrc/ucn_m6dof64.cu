// Kernel instantiations: 14-state 6-DOF Mars landing, FP64 plain path.  The fused solve
// with global-memory records and the stand-alone ADMM compile in their own
// units (ucn_m6dof64_*.cu).
#include "ucn_launch.cuh"
UCN_EXTERN_SCP(Mars14, double, false, false)
UCN_EXTERN_ADMM(Mars14, double, true, false)
UCN_EXTERN_ADMM(Mars14, double, false, false)
UCN_DEFINE_LAUNCHERS(m6dof64, Mars14, double, false)
