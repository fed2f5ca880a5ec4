// Kernel instantiation: scenario groups of the 12-state quadrotor on the lane
// layout (thread-block clusters, one CTA per scenario, 4 threads per node), FP64 plain path.
#include "ucn_launch.cuh"
UCN_DEFINE_GROUP_LANES(Quad12, double, false)
