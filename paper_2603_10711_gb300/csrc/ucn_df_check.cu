// ucn_df_check: the FP32 path's double-float arithmetic on given inputs, so
// that it can be checked against FP64 (a diagnostic entry point).
#include <cuda_runtime.h>

#include "ucn_internal.h"
#include "ucn_math.cuh"

using namespace ucn;

namespace {

__global__ void df_op_kernel(int op, const double* a, const double* b, long long n, double* out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const DF x = df_from(a[k]);
  const DF y = (op == UCN_DF_SQRT || op == UCN_DF_ROUND) ? DF() : df_from(b[k]);
  DF r;
  switch (op) {
    case UCN_DF_ADD: r = df_add(x, y); break;
    case UCN_DF_SUB: r = df_sub(x, y); break;
    case UCN_DF_MUL: r = df_mul(x, y); break;
    case UCN_DF_DIV: r = df_div(x, y); break;
    case UCN_DF_SQRT: r = df_sqrt(x); break;
    default: r = x; break;
  }
  out[k] = df_to_double(r);
}

// The residual accumulation of the FP32 path on given data: one thread sums
// (float(a_k) - float(b_k))^2 (or float(a_k)^2) over k in order.
__global__ void df_sum_kernel(int op, const double* a, const double* b, long long n, double* out) {
  DF acc;
  for (long long k = 0; k < n; ++k) {
    if (op == UCN_DF_SQDIFF_SUM) acc_sq_diff(acc, __double2float_rn(a[k]), __double2float_rn(b[k]));
    else acc_sq(acc, __double2float_rn(a[k]));
  }
  out[0] = df_to_double(acc);
}

template <class M>
__global__ void df_rk4_kernel(const double* x, const double* u, const double* prm, double h, long long n, double* out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  constexpr int NX = M::NX, NU = M::NU;
  DF p[8], xs[NX], us[NU], xn[NX];
  for (int j = 0; j < 8; ++j) p[j] = df_from(prm[j]);
  for (int j = 0; j < NX; ++j) xs[j] = df_from(x[k * NX + j]);
  for (int j = 0; j < NU; ++j) us[j] = df_from(u[k * NU + j]);
  rk4h<M, DF, DF, DF>(p, df_from(h), df_from(0.5 * h), df_from(h / 6.0), xs, us, xn);
  for (int j = 0; j < NX; ++j) out[k * NX + j] = df_to_double(xn[j]);
}

}  // namespace

extern "C" ucn_status ucn_df_check(int op, const double* a_d, const double* b_d, const double* prm_d, double h,
                                   long long n, double* out_d, void* stream) {
  set_error_message("");
  if (n < 0 || !out_d || !a_d) { set_error_message("null argument or n < 0"); return UCN_EINVAL; }
  if (n == 0) return UCN_OK;
  const cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (op >= UCN_DF_ADD && op <= UCN_DF_ROUND) {
    if (!b_d && op != UCN_DF_SQRT && op != UCN_DF_ROUND) { set_error_message("null argument"); return UCN_EINVAL; }
    df_op_kernel<<<blocks, 128, 0, st>>>(op, a_d, b_d, n, out_d);
  } else if (op == UCN_DF_SQDIFF_SUM || op == UCN_DF_SQ_SUM) {
    if (!b_d && op == UCN_DF_SQDIFF_SUM) { set_error_message("null argument"); return UCN_EINVAL; }
    df_sum_kernel<<<1, 1, 0, st>>>(op, a_d, b_d, n, out_d);
  } else if (op > UCN_DF_RK4 && model_known(op - UCN_DF_RK4)) {
    if (!b_d || !prm_d) { set_error_message("null argument"); return UCN_EINVAL; }
    switch (op - UCN_DF_RK4) {
      case UCN_MODEL_QUAD12: df_rk4_kernel<Quad12><<<blocks, 128, 0, st>>>(a_d, b_d, prm_d, h, n, out_d); break;
      case UCN_MODEL_QUAT13: df_rk4_kernel<Quat13><<<blocks, 128, 0, st>>>(a_d, b_d, prm_d, h, n, out_d); break;
      case UCN_MODEL_MARS14: df_rk4_kernel<Mars14><<<blocks, 128, 0, st>>>(a_d, b_d, prm_d, h, n, out_d); break;
      default: df_rk4_kernel<Mars7><<<blocks, 128, 0, st>>>(a_d, b_d, prm_d, h, n, out_d); break;
    }
  } else {
    set_error_message("unknown double-float check op");
    return UCN_EINVAL;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error_message(cudaGetErrorString(e)); return UCN_ECUDA; }
  return UCN_OK;
}
