// Kernel instantiation: 12-state quadrotor, FP32 path with refinement, fused solve on the lane
// layout (4 threads per node) with node records in shared memory;
// CTAs of up to 512 threads, 128 registers per thread.
#include "ucn_launch.cuh"
UCN_INSTANTIATE_SCPL(Quad12, float, true, true, ucn::LANES_MAX_THREADS)
