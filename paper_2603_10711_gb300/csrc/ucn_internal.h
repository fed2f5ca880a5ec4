// Host-side internals shared by the C-ABI implementation and the per-model
// launch units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "ucn.h"

namespace ucn {

struct ProblemDev;
struct Layout;

// Sets the thread-local message returned by ucn_last_error (ucn_api.cu).
void set_error_message(const char* msg);

// Host-side fault injection: with UCN_FAULT_ALLOC=n in the environment the
// n-th device or pinned allocation (1-based) of a ucn_problem_create or
// ucn_serve_create call fails as if the memory were exhausted; 0 when unset.
int fault_alloc_at();

// Node-record layout of one instance for a kernel with `tpn` threads per node
// (defined in ucn_api.cu).
Layout make_layout(int model, int nodes, int max_obs, int tsize, bool reg_mats, int tpn);

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
  int tpn;              // threads per node of the fused solve: 1; 2 (pair kernel: 3-DOF Mars, FP32,
                        // records in shared memory); 4 (lane kernel, quadrotor)
  int* launched = nullptr;   // out (when not NULL): kernel launches the fused solve made
};

// Threads per node the fused solve uses by default for a model, node count and
// precision (records in shared memory; 1 otherwise for the 3-DOF Mars model).
int default_tpn(int model, int nodes, int precision);
// Whether `tpn` threads per node can run a model, node count and precision
// (with the node records in shared memory when smem).
bool tpn_allowed(int tpn, int model, int nodes, int precision, bool smem);

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
UCN_DECLARE_LAUNCHERS(quat64)
UCN_DECLARE_LAUNCHERS(quat32)
UCN_DECLARE_LAUNCHERS(m6dof64)
UCN_DECLARE_LAUNCHERS(m6dof32)

// Model properties used by the host code.
inline bool model_known(int m) {
  return m == UCN_MODEL_QUAD12 || m == UCN_MODEL_MARS7 || m == UCN_MODEL_QUAT13 || m == UCN_MODEL_MARS14;
}
inline int model_nx(int m) {
  return m == UCN_MODEL_QUAD12 ? 12 : m == UCN_MODEL_QUAT13 ? 13 : m == UCN_MODEL_MARS14 ? 14 : 7;
}
inline int model_nu(int m) { return (m == UCN_MODEL_MARS7 || m == UCN_MODEL_MARS14) ? 3 : 4; }
// quadrotors: obstacle mirrors; Mars models: their thrust / attitude / glide-slope sets
inline bool model_obstacles(int m) { return m == UCN_MODEL_QUAD12 || m == UCN_MODEL_QUAT13; }

// Penalty factor of each SCP iteration, (rho_final / rho_geo)^(k / (K - 1))
// (1 without a schedule), tabulated on the host so that no kernel evaluates
// pow per iteration.
std::vector<double> rho_schedule(double rho_final, double rho_geo, int K);
// Entry k of that schedule.
double rho_factor(double rho_final, double rho_geo, int K, int k);

// The launchers of one model and precision.
struct Launchers {
  cudaError_t (*scp)(const LaunchCfg&, const double*, const double*, double*, double*, ucn_scp_stats*, int*);
  cudaError_t (*admm)(const LaunchCfg&, const double*, const double*, const double*, const double*, const double*,
                      const double*, int, int, double*, double*, double*, int*);
  cudaError_t (*linearize)(const void*, const int*, long long, const double*, const double*, double*, double*,
                           double*, cudaStream_t);
};
inline Launchers launchers_for(int model, int precision) {
  const bool f64 = precision == UCN_PREC_FP64;
  if (model == UCN_MODEL_QUAD12) return f64 ? Launchers{quad64_scp, quad64_admm, quad64_linearize}
                                            : Launchers{quad32_scp, quad32_admm, quad32_linearize};
  if (model == UCN_MODEL_QUAT13) return f64 ? Launchers{quat64_scp, quat64_admm, quat64_linearize}
                                            : Launchers{quat32_scp, quat32_admm, quat32_linearize};
  if (model == UCN_MODEL_MARS14) return f64 ? Launchers{m6dof64_scp, m6dof64_admm, m6dof64_linearize}
                                            : Launchers{m6dof32_scp, m6dof32_admm, m6dof32_linearize};
  return f64 ? Launchers{mars64_scp, mars64_admm, mars64_linearize} : Launchers{mars32_scp, mars32_admm, mars32_linearize};
}

// The device-resident request loop of a server (ucn_serve.cuh), one launcher
// per model and precision; NULL for an unknown model.
struct LoopCfg;
cudaError_t quad64_loop(const LoopCfg& c);
cudaError_t quad32_loop(const LoopCfg& c);
cudaError_t mars64_loop(const LoopCfg& c);
cudaError_t mars32_loop(const LoopCfg& c);
cudaError_t quat64_loop(const LoopCfg& c);
cudaError_t quat32_loop(const LoopCfg& c);
cudaError_t m6dof64_loop(const LoopCfg& c);
cudaError_t m6dof32_loop(const LoopCfg& c);
inline cudaError_t (*loop_launcher_for(int model, int precision))(const LoopCfg&) {
  const bool f64 = precision == UCN_PREC_FP64;
  if (model == UCN_MODEL_QUAD12) return f64 ? quad64_loop : quad32_loop;
  if (model == UCN_MODEL_MARS7) return f64 ? mars64_loop : mars32_loop;
  if (model == UCN_MODEL_QUAT13) return f64 ? quat64_loop : quat32_loop;
  if (model == UCN_MODEL_MARS14) return f64 ? m6dof64_loop : m6dof32_loop;
  return nullptr;
}

// Scenario groups (quadrotor only): thread-block clusters, one CTA per scenario.
cudaError_t quad64_scp_group(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                             ucn_scp_stats* st, int* status);
cudaError_t quad32_scp_group(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                             ucn_scp_stats* st, int* status);

}  // namespace ucn
