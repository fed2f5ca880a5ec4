// Device-resident request loop of a server: 13-state quaternion quadrotor, FP64 plain path; one thread
// per node, node records in shared memory here, the other variant in its own unit (compiled in
// parallel).
#include "ucn_launch.cuh"
#include "ucn_serve.cuh"
UCN_EXTERN_LOOP(Quat13, double, false, false, 1)
UCN_INSTANTIATE_LOOP(Quat13, double, true, false, 1)
UCN_DEFINE_LOOP_LAUNCHER(quat64, Quat13, double, false)
