// Device-resident request loop of a server: 3-DOF Mars descent, FP64 plain path; one thread per node,
// node records in shared memory here, the other variants in their own units (compiled in parallel).
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_EXTERN_LOOP(Mars7, double, false, false, 1)
UCN_INSTANTIATE_LOOP(Mars7, double, true, false, 1)
UCN_DEFINE_LOOP_LAUNCHER(mars64, Mars7, double, false)
