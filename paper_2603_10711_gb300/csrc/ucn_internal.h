// Host-side internals shared by the C-ABI implementation and the per-model
// launch units.
#pragma once
#include <cuda_runtime.h>

#include "ucn.h"

namespace ucn {

struct ProblemDev;
struct Layout;

// Sets the thread-local message returned by ucn_last_error (ucn_api.cu).
void set_error_message(const char* msg);

// Node-record layout of one instance (defined in ucn_api.cu).
Layout make_layout(int model, int nodes, int max_obs, int tsize, bool reg_mats);

// Everything one kernel launch needs besides its buffers.
struct LaunchCfg {
  const void* P;        // ProblemDev*
  const void* L;        // Layout*
  bool smem;            // per-node arrays in shared memory (else the global workspace)
  long long smem_bytes; // dynamic shared memory per CTA when smem
  int threads;          // CTA size
  int blocks;           // one CTA per instance
  cudaStream_t stream;
  int group;            // CTAs per thread-block cluster (scenario groups only)
  int nodes;            // nodes of the longest instance (N_max + 1)
  int tpn;              // threads per node of the fused solve: 1, or 4 (lane kernel, quadrotor)
};

// Threads per node the fused solve uses by default for a model and node count.
int default_tpn(int model, int nodes);

// Launchers, one translation unit per (model, precision) so that the four
// compile in parallel.
#define UCN_DECLARE_LAUNCHERS(NAME)                                                                    \
  cudaError_t NAME##_scp(const LaunchCfg& c, const double* x0, const double* u0, double* xo,          \
                         double* uo, ucn_scp_stats* st, int* status);                                 \
  cudaError_t NAME##_admm(const LaunchCfg& c, const double* xbar, const double* ubar,                 \
                          const double* A, const double* B, const double* d, const double* radius,    \
                          int iters, int warm, double* xhat, double* uhat, double* res, int* status); \
  cudaError_t NAME##_linearize(const void* P, const int* node_inst, long long total_u,                \
                               const double* xbar, const double* ubar, double* A, double* B,          \
                               double* d, cudaStream_t stream);
UCN_DECLARE_LAUNCHERS(quad64)
UCN_DECLARE_LAUNCHERS(quad32)
UCN_DECLARE_LAUNCHERS(mars64)
UCN_DECLARE_LAUNCHERS(mars32)

// Scenario groups (quadrotor only): thread-block clusters, one CTA per scenario.
cudaError_t quad64_scp_group(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                             ucn_scp_stats* st, int* status);
cudaError_t quad32_scp_group(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                             ucn_scp_stats* st, int* status);

}  // namespace ucn
