// Kernel instantiation: scenario groups of the 12-state quadrotor (thread-block
// clusters, one CTA per scenario), FP64 path.
#include "ucn_launch.cuh"
UCN_DEFINE_GROUP_LAUNCHER(quad64, Quad12, double, false)
