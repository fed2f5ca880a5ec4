// Launch wrappers, instantiated once per model by ucn_quad.cu / ucn_mars.cu.
#pragma once
#include "ucn_internal.h"
#include "ucn_kernels.cuh"

namespace ucn {

template <class M, class T, bool R>
cudaError_t launch_scp_t(const LaunchCfg& c, const double* x0, const double* u0, double* xo, double* uo,
                         ucn_scp_stats* st, int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  if (c.smem) {
    auto k = scp_kernel<M, T, true, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
    k<<<c.blocks, c.threads, c.smem_bytes, c.stream>>>(P, L, x0, u0, xo, uo, st, status);
  } else {
    scp_kernel<M, T, false, R><<<c.blocks, c.threads, 0, c.stream>>>(P, L, x0, u0, xo, uo, st, status);
  }
  return cudaGetLastError();
}

template <class M, class T, bool R>
cudaError_t launch_admm_t(const LaunchCfg& c, const double* xbar, const double* ubar, const double* A,
                          const double* B, const double* d, const double* radius, int iters, int warm,
                          double* xhat, double* uhat, double* res, int* status) {
  const ProblemDev& P = *(const ProblemDev*)c.P;
  const Layout& L = *(const Layout*)c.L;
  if (c.smem) {
    auto k = admm_kernel<M, T, true, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
    k<<<c.blocks, c.threads, c.smem_bytes, c.stream>>>(P, L, xbar, ubar, A, B, d, radius, iters, warm, xhat, uhat,
                                                      res, status);
  } else {
    admm_kernel<M, T, false, R><<<c.blocks, c.threads, 0, c.stream>>>(P, L, xbar, ubar, A, B, d, radius, iters, warm,
                                                                      xhat, uhat, res, status);
  }
  return cudaGetLastError();
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
