// Kernel instantiation: scenario groups of the 12-state quadrotor (thread-block
// clusters, one CTA per scenario), FP32 path with refinement.
#include "ucn_launch.cuh"
UCN_DEFINE_GROUP_LAUNCHER(quad32, Quad12, float, true)
