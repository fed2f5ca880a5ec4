// Kernel instantiation: scenario groups of the 12-state quadrotor on the lane
// layout (thread-block clusters, one CTA per scenario, 4 threads per node), FP32 path with refinement;
// CTAs of up to 512 threads, 128 registers per thread.
#include "ucn_launch.cuh"
UCN_DEFINE_GROUP_LANES(Quad12, float, true, ucn::LANES_MAX_THREADS)
