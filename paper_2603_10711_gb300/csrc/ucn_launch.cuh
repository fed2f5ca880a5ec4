// Launch wrappers, instantiated per (model, precision) by the ucn_<model><bits>*.cu units.
#pragma once
#include "ucn_internal.h"
#include "ucn_kernels.cuh"
#include "ucn_lanes.cuh"
#include "ucn_pair.cuh"

namespace ucn {

// The 3-CTAs-per-SM variant of the one-thread kernel (scp_kernel_3): set-up,
// occupancy and launch, explicitly instantiated in its own translation unit
// for the configurations listed in has_scp3.
template <class M, class T, bool SMEM, bool R>
constexpr bool has_scp3 = false;
template <>
constexpr bool has_scp3<Mars7, float, true, true> = true;

template <class M, class T, bool SMEM, bool R>
struct Scp3Variant {
  static cudaError_t occupancy(const LaunchCfg& c, int* blocks);
  static cudaError_t launch(const LaunchCfg& c, const ProblemDev& P, int blocks, const double* x0, const double* u0,
                            double* xo, double* uo, ucn_scp_stats* st, int* status);
};
// (defined out of the class, so that an extern template declaration keeps the
// kernel out of the translation units that only launch it)
template <class M, class T, bool SMEM, bool R>
cudaError_t Scp3Variant<M, T, SMEM, R>::occupancy(const LaunchCfg& c, int* blocks) {
  *blocks = 0;
  if (c.threads > SCP3_MAX_THREADS) return cudaSuccess;
  auto k = scp_kernel_3<M, T, SMEM, R>;
  if (SMEM) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, c.threads, SMEM ? c.smem_bytes : 0);
}
template <class M, class T, bool SMEM, bool R>
cudaError_t Scp3Variant<M, T, SMEM, R>::launch(const LaunchCfg& c, const ProblemDev& P, int blocks, const double* x0,
                                               const double* u0, double* xo, double* uo, ucn_scp_stats* st,
                                               int* status) {
  const Layout& L = *(const Layout*)c.L;
  auto k = scp_kernel_3<M, T, SMEM, R>;
  if (SMEM) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  k<<<blocks, c.threads, SMEM ? c.smem_bytes : 0, c.stream>>>(P, L, x0, u0, xo, uo, st, status);
  return cudaGetLastError();
}

// Time of one CTA of scp_kernel_3 (three per SM) over one of scp_kernel (two
// per SM), measured on the Mars batch (6.78 vs 4.66 ms per instance, GB300).
constexpr double SCP3_TIME_RATIO = 1.45;

// How many of a launch's CTAs (taken in the launch's order) run as
// scp_kernel_3 before the rest run as scp_kernel: the split with the shortest
// modelled time, rounds(k3 on b3 per SM) x SCP3_TIME_RATIO + rounds(rest on b2
// per SM).  Whole CTAs are resident in rounds, so a batch that is not a whole
// number of rounds leaves SMs idle in its last one; one round of three CTAs per
// SM followed by rounds of two fills 1024 CTAs on 152 SMs in 3.4 round-times
// instead of 4.  0 when the variant keeps no more CTAs resident.
inline int scp3_split(int B, int sms, int b2, int b3) {
  if (b3 <= b2 || b2 < 1 || sms < 1) return 0;
  const long long r2 = (long long)sms * b2, r3 = (long long)sms * b3;
  auto cost = [&](long long k3) {
    return (double)((k3 + r3 - 1) / r3) * SCP3_TIME_RATIO + (double)((B - k3 + r2 - 1) / r2);
  };
  long long best = 0;
  double bc = cost(0);
  for (long long k3 = r3;; k3 += r3) {
    const long long k = k3 < B ? k3 : B;
    const double v = cost(k);
    if (v < bc - 1e-9) { bc = v; best = k; }
    if (k3 >= B) break;
  }
  return (int)best;
}

// One kernel variant per function, so that a translation unit can leave a
// variant to another one (extern template) and the slow ones compile in parallel.
template <class M, class T, bool SMEM, bool R>
cudaError_t launch_scp_v(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                         ucn_scp_stats* st, int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  auto k = scp_kernel<M, T, SMEM, R>;
  if (SMEM) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  int k3 = 0;
  if constexpr (has_scp3<M, T, SMEM, R>) {
    // the first k3 CTAs of the order on the 3-per-SM variant, the rest after them
    if (P.order && c.threads <= SCP3_MAX_THREADS && c.blocks > 0) {
      int dev = 0, sms = 0, b2 = 0, b3 = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k, c.threads, SMEM ? c.smem_bytes : 0);
      if (e == cudaSuccess) e = Scp3Variant<M, T, SMEM, R>::occupancy(c, &b3);
      if (e != cudaSuccess) return e;
      k3 = scp3_split(c.blocks, sms, b2, b3);
      if (k3 > 0) {
        e = Scp3Variant<M, T, SMEM, R>::launch(c, P, k3, x0, u0, xo, uo, st, status);
        if (e != cudaSuccess) return e;
      }
    }
  }
  if (c.launched) *c.launched = (k3 > 0) + (k3 < c.blocks);
  if (k3 >= c.blocks) return cudaSuccess;
  ProblemDev Pr = P;
  if (k3 > 0) Pr.order = P.order + k3;
  k<<<c.blocks - k3, c.threads, SMEM ? c.smem_bytes : 0, c.stream>>>(Pr, L, x0, u0, xo, uo, st, status);
  return cudaGetLastError();
}

// The lane kernel (4 threads per node; quadrotor), one register class per
// variant (MAXT: LANES_WIDE_THREADS or LANES_MAX_THREADS): set-up, occupancy
// and launch, explicitly instantiated in one translation unit per variant.
template <class M, class T, bool SMEM, bool R, int MAXT>
struct LanesVariant {
  // CTAs of `threads` threads and the layout's shared memory resident per SM (0: none)
  static cudaError_t occupancy(const LaunchCfg& c, int threads, int* blocks);
  static cudaError_t launch(const LaunchCfg& c, int threads, const double* x0, const double* u0, double* xo,
                            double* uo, ucn_scp_stats* st, int* status);
};
// (defined out of the class, so that an extern template declaration keeps the
// kernel out of the translation units that only launch it)
template <class M, class T, bool SMEM, bool R, int MAXT>
cudaError_t LanesVariant<M, T, SMEM, R, MAXT>::occupancy(const LaunchCfg& c, int threads, int* blocks) {
  *blocks = 0;
  if (threads > MAXT) return cudaSuccess;
  auto k = lanes_kernel<M, T, SMEM, R, false, 4, MAXT>();
  if (SMEM) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, threads, SMEM ? c.smem_bytes : 0);
}
template <class M, class T, bool SMEM, bool R, int MAXT>
cudaError_t LanesVariant<M, T, SMEM, R, MAXT>::launch(const LaunchCfg& c, int threads, const double* x0,
                                                      const double* u0, double* xo, double* uo, ucn_scp_stats* st,
                                                      int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  if (threads > MAXT) return cudaErrorInvalidConfiguration;
  auto k = lanes_kernel<M, T, SMEM, R, false, 4, MAXT>();
  if (SMEM) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  k<<<c.blocks, threads, SMEM ? c.smem_bytes : 0, c.stream>>>(P, L, x0, u0, xo, uo, st, status);
  return cudaGetLastError();
}

// Whether the wide-register variant keeps at least as many CTAs of this launch
// resident per SM as the 128-register one (then it runs without the spills).
template <class Wide, class Narrow>
cudaError_t lanes_prefer_wide(const LaunchCfg& c, int threads, bool* wide) {
  *wide = false;
  if (threads > LANES_WIDE_THREADS) return cudaSuccess;
  int bw = 0, bn = 0;
  cudaError_t e = Wide::occupancy(c, threads, &bw);
  if (e == cudaSuccess) e = Narrow::occupancy(c, threads, &bn);
  if (e != cudaSuccess) return e;
  *wide = bw > 0 && bw >= bn;
  return cudaSuccess;
}

template <class M, class T, bool SMEM, bool R>
cudaError_t launch_scpl_v(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                          ucn_scp_stats* st, int* status) {
  using Wide = LanesVariant<M, T, SMEM, R, LANES_WIDE_THREADS>;
  using Narrow = LanesVariant<M, T, SMEM, R, LANES_MAX_THREADS>;
  const int threads = (4 * c.nodes + 31) / 32 * 32;
  if (threads > LANES_MAX_THREADS) return cudaErrorInvalidConfiguration;
  bool wide = false;
  cudaError_t e = lanes_prefer_wide<Wide, Narrow>(c, threads, &wide);
  if (e != cudaSuccess) return e;
  return wide ? Wide::launch(c, threads, x0, u0, xo, uo, st, status)
              : Narrow::launch(c, threads, x0, u0, xo, uo, st, status);
}

// The pair kernel (2 threads per node; 3-DOF Mars, FP32, records in shared memory).
template <class M, bool R>
cudaError_t launch_scpp_v(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                          ucn_scp_stats* st, int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  auto k = scp_kernel_pair<M, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
  if (e != cudaSuccess) return e;
  // the whole unified L1 / shared memory as shared memory: two ~105 KB CTAs per SM
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  const int threads = (2 * c.nodes + 31) / 32 * 32;
  if (!c.smem || threads > PAIR_MAX_THREADS) return cudaErrorInvalidConfiguration;
  k<<<c.blocks, threads, c.smem_bytes, c.stream>>>(P, L, x0, u0, xo, uo, st, status);
  return cudaGetLastError();
}

template <class M, class T, bool R>
cudaError_t launch_scp_t(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                         ucn_scp_stats* st, int* status) {
  if constexpr (std::is_same<M, Mars7>::value && std::is_same<T, float>::value && R) {
    if (c.tpn == 2) return launch_scpp_v<M, R>(c, x0, u0, xo, uo, st, status);
  }
  if constexpr (LaneModel<M>::value) {
    if (c.tpn == 4)
      return c.smem ? launch_scpl_v<M, T, true, R>(c, x0, u0, xo, uo, st, status)
                    : launch_scpl_v<M, T, false, R>(c, x0, u0, xo, uo, st, status);
  }
  return c.smem ? launch_scp_v<M, T, true, R>(c, x0, u0, xo, uo, st, status)
                : launch_scp_v<M, T, false, R>(c, x0, u0, xo, uo, st, status);
}

// The group kernels of the lane layout, one per register class (each in its
// own translation unit: defined there).
template <class M, class T, bool R>
using ScpKernelPtr = void (*)(ProblemDev, Layout, const double*, const double*, double*, double*, ucn_scp_stats*, int*);
template <class M, class T, bool R, int MAXT>
ScpKernelPtr<M, T, R> scp_group_lanes();

// The group lane kernel for CTAs of `threads` threads: the wide-register
// variant when it keeps as many CTAs resident per SM.
template <class M, class T, bool R>
cudaError_t pick_group_lanes(const LaunchCfg& c, int threads, ScpKernelPtr<M, T, R>* out) {
  auto kw = scp_group_lanes<M, T, R, LANES_WIDE_THREADS>();
  auto kn = scp_group_lanes<M, T, R, LANES_MAX_THREADS>();
  *out = kn;
  if (threads > LANES_WIDE_THREADS) return cudaSuccess;
  int bw = 0, bn = 0;
  for (auto k : {kw, kn}) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, kw, threads, c.smem_bytes);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bn, kn, threads, c.smem_bytes);
  if (e != cudaSuccess) return e;
  if (bw > 0 && bw >= bn) *out = kw;
  return cudaSuccess;
}

// Scenario groups: thread-block clusters of c.group CTAs (records in shared
// memory only), P.gclusters clusters per group.  cudaErrorInvalidClusterSize
// when fewer than the clusters of one group can be resident together (cluster
// size above 16, or too much shared memory per CTA).
template <class M, class T, bool R>
cudaError_t launch_scp_group_t(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                               ucn_scp_stats* st, int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  if (!c.smem || c.group < 1 || c.group > 16 || c.blocks % c.group) return cudaErrorInvalidClusterSize;
  const int threads = c.tpn == 4 ? (4 * c.nodes + 31) / 32 * 32 : c.threads;
  if (threads > LANES_MAX_THREADS) return cudaErrorInvalidConfiguration;
  ScpKernelPtr<M, T, R> k = scp_kernel<M, T, true, R, true>;
  cudaError_t e = cudaSuccess;
  if (c.tpn == 4) {
    e = pick_group_lanes<M, T, R>(c, threads, &k);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
  if (e != cudaSuccess) return e;
  if (c.group > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c.blocks, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)c.smem_bytes;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)c.group;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < (P.gclusters > 1 ? P.gclusters : 1)) return cudaErrorInvalidClusterSize;
  return cudaLaunchKernelEx(&cfg, k, P, L, x0, u0, xo, uo, st, status);
}

template <class M, class T, bool SMEM, bool R>
cudaError_t launch_admm_v(const LaunchCfg& c, const double* xbar, const double* ubar, const double* A,
                          const double* B, const double* d, const double* radius, int iters, int warm,
                          double* xhat, double* uhat, double* res, int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  auto k = admm_kernel<M, T, SMEM, R>;
  if (SMEM) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  k<<<c.blocks, c.threads, SMEM ? c.smem_bytes : 0, c.stream>>>(P, L, xbar, ubar, A, B, d, radius, iters, warm,
                                                                xhat, uhat, res, status);
  return cudaGetLastError();
}

template <class M, class T, bool R>
cudaError_t launch_admm_t(const LaunchCfg& c, const double* xbar, const double* ubar, const double* A,
                          const double* B, const double* d, const double* radius, int iters, int warm,
                          double* xhat, double* uhat, double* res, int* status) {
  return c.smem ? launch_admm_v<M, T, true, R>(c, xbar, ubar, A, B, d, radius, iters, warm, xhat, uhat, res, status)
                : launch_admm_v<M, T, false, R>(c, xbar, ubar, A, B, d, radius, iters, warm, xhat, uhat, res, status);
}

template <class M, class T>
cudaError_t launch_linearize_t(const void* Pv, const int* node_inst, long long total_u, const double* xbar,
                               const double* ubar, double* A, double* B, double* d, cudaStream_t stream) {
  const ProblemDev& P = *(const ProblemDev*)Pv;
  const int threads = 128;
  const long long blocks = (total_u + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  linearize_kernel<M, T><<<(unsigned)blocks, threads, 0, stream>>>(P, node_inst, total_u, xbar, ubar, A, B, d);
  return cudaGetLastError();
}

}  // namespace ucn

// FP64: plain path (no refinement); FP32: refinement on every KKT solve.
#define UCN_DEFINE_LAUNCHERS(NAME, MODEL, T, REFINE)                                                       \
  namespace ucn {                                                                                          \
  cudaError_t NAME##_scp(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,   \
                         ucn_scp_stats* st, int* status) {                                                 \
    return launch_scp_t<MODEL, T, REFINE>(c, x0, u0, xo, uo, st, status);                                 \
  }                                                                                                        \
  cudaError_t NAME##_admm(const LaunchCfg& c, const double* xbar, const double* ubar, const double* A,     \
                          const double* B, const double* d, const double* radius, int iters, int warm,    \
                          double* xhat, double* uhat, double* res, int* status) {                         \
    return launch_admm_t<MODEL, T, REFINE>(c, xbar, ubar, A, B, d, radius, iters, warm, xhat, uhat, res,  \
                                           status);                                                        \
  }                                                                                                        \
  cudaError_t NAME##_linearize(const void* P, const int* node_inst, long long total_u, const double* xbar, \
                               const double* ubar, double* A, double* B, double* d, cudaStream_t stream) { \
    return launch_linearize_t<MODEL, T>(P, node_inst, total_u, xbar, ubar, A, B, d, stream);              \
  }                                                                                                        \
  }

// Scenario-group solve, one translation unit per (model, precision).
#define UCN_DEFINE_GROUP_LAUNCHER(NAME, MODEL, T, REFINE)                                                 \
  namespace ucn {                                                                                          \
  cudaError_t NAME##_scp_group(const LaunchCfg& c, const double* x0, const double* u0, double* xo,         \
                               double* uo, ucn_scp_stats* st, int* status) {                               \
    return launch_scp_group_t<MODEL, T, REFINE>(c, x0, u0, xo, uo, st, status);                           \
  }                                                                                                        \
  }

// Explicit instantiation of one kernel variant (SMEM: records in shared memory)
// in its own translation unit; the UCN_EXTERN_* forms keep it out of the others.
#define UCN_SCP_V(MODEL, T, SMEM, REFINE)                                                                  \
  cudaError_t ucn::launch_scp_v<ucn::MODEL, T, SMEM, REFINE>(const ucn::LaunchCfg&, const double*,       \
                                                             const double*, double*, double*,            \
                                                             ucn_scp_stats*, int*)
#define UCN_ADMM_V(MODEL, T, SMEM, REFINE)                                                                 \
  cudaError_t ucn::launch_admm_v<ucn::MODEL, T, SMEM, REFINE>(                                           \
      const ucn::LaunchCfg&, const double*, const double*, const double*, const double*, const double*,  \
      const double*, int, int, double*, double*, double*, int*)
#define UCN_INSTANTIATE_SCP(MODEL, T, SMEM, REFINE) template UCN_SCP_V(MODEL, T, SMEM, REFINE);
#define UCN_INSTANTIATE_ADMM(MODEL, T, SMEM, REFINE) template UCN_ADMM_V(MODEL, T, SMEM, REFINE);
#define UCN_EXTERN_SCP(MODEL, T, SMEM, REFINE) extern template UCN_SCP_V(MODEL, T, SMEM, REFINE);
#define UCN_EXTERN_ADMM(MODEL, T, SMEM, REFINE) extern template UCN_ADMM_V(MODEL, T, SMEM, REFINE);

// Lane-kernel variants (records in shared or global memory, register class
// MAXT), each in its own translation unit.
#define UCN_INSTANTIATE_SCPL(MODEL, T, SMEM, REFINE, MAXT) template struct ucn::LanesVariant<ucn::MODEL, T, SMEM, REFINE, MAXT>;
#define UCN_EXTERN_SCPL(MODEL, T, SMEM, REFINE, MAXT) extern template struct ucn::LanesVariant<ucn::MODEL, T, SMEM, REFINE, MAXT>;
#define UCN_DEFINE_GROUP_LANES(MODEL, T, REFINE, MAXT)                                                     \
  namespace ucn {                                                                                          \
  template <>                                                                                              \
  ScpKernelPtr<MODEL, T, REFINE> scp_group_lanes<MODEL, T, REFINE, MAXT>() {                               \
    return lanes_kernel<MODEL, T, true, REFINE, true, 4, MAXT>();                                          \
  }                                                                                                        \
  }

// The 3-CTAs-per-SM variant of the one-thread kernel in its own translation unit.
#define UCN_INSTANTIATE_SCP3(MODEL, T, SMEM, REFINE) template struct ucn::Scp3Variant<ucn::MODEL, T, SMEM, REFINE>;
#define UCN_EXTERN_SCP3(MODEL, T, SMEM, REFINE) extern template struct ucn::Scp3Variant<ucn::MODEL, T, SMEM, REFINE>;

// Pair-kernel variant in its own translation unit.
#define UCN_SCPP_V(MODEL, REFINE)                                                                          \
  cudaError_t ucn::launch_scpp_v<ucn::MODEL, REFINE>(const ucn::LaunchCfg&, const double*, const double*, \
                                                     double*, double*, ucn_scp_stats*, int*)
#define UCN_INSTANTIATE_SCPP(MODEL, REFINE) template UCN_SCPP_V(MODEL, REFINE);
#define UCN_EXTERN_SCPP(MODEL, REFINE) extern template UCN_SCPP_V(MODEL, REFINE);
