// Kernel instantiation: scenario groups of the 12-state quadrotor on the lane
// layout (thread-block clusters, one CTA per scenario, 4 threads per node), plain FP64 path;
// CTAs of up to 384 threads, 168 registers per thread.
#include "ucn_launch.cuh"
UCN_DEFINE_GROUP_LANES(Quad12, double, false, ucn::LANES_WIDE_THREADS)
