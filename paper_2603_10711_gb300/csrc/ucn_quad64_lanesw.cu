// Kernel instantiation: 12-state quadrotor, plain FP64 path, fused solve on the lane
// layout (4 threads per node) with node records in shared memory;
// CTAs of up to 384 threads, 168 registers per thread.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCPL(Quad12, double, true, false, ucn::LANES_WIDE_THREADS)
