// Kernel instantiation: 12-state quadrotor, plain FP64 path, fused solve on the lane
// layout (4 threads per node) with node records in global memory;
// CTAs of up to 512 threads, 128 registers per thread.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCPL(Quad12, double, false, false, ucn::LANES_MAX_THREADS)
