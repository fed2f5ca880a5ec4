// ucn_scp_solve_noalloc: the fused SCP solve for callers that cannot
// allocate device memory.
//
// Who needs it.  ucn_problem_create allocates the problem's device copy and
// workspace with cudaMalloc.  Some callers cannot: code that runs inside a
// real-time control loop where allocation (and its implicit device
// synchronisation) is forbidden, an application whose memory pool owns the
// whole GPU, or a runtime that hands us pre-registered buffers only.  They
// already hold their problem data on the device, so this entry point takes
// the descriptor's arrays as device pointers and keeps the kernel's scratch
// (per-instance index tables and the final ADMM state the kernel writes out)
// in one file-scope __device__ array instead of allocated memory.
//
// Limits and sharing.  The array (index tables, the penalty schedule, the
// exported state) holds UCN_NOALLOC_SCRATCH_BYTES (64 MiB) on
// every GPU that loads the library, until the process exits.  The tables reach
// it through small set-up kernels that take them as by-value parameters, so
// the call copies nothing from host memory and does not wait for the stream.  All calls share
// it and it keeps the last call's contents; two calls whose kernels overlap on
// the GPU (different streams, or different host threads on one device) race
// on it.  Nothing in it has to start at zero: each call writes every table
// entry and every exported state entry its kernel reads or reports.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ucn_internal.h"
#include "ucn_kernels.cuh"

using namespace ucn;

static __device__ __align__(256) unsigned char g_noalloc_scratch[UCN_NOALLOC_SCRATCH_BYTES];

namespace {

ucn_status nfail(ucn_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_error_message(buf);
  return s;
}

long long up256(long long v) { return (v + 255) / 256 * 256; }

// Device address of the scratch array, looked up once per device with that
// device current (a host-side name of a __device__ variable is not a device
// address).
std::mutex g_mu;
void* g_addr[128] = {nullptr};

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// The index tables and the penalty schedule reach the device as kernel
// parameters (copied into the launch by value, 4 KB or less each), not by a
// copy from host memory: a copy from pageable memory would make the call wait
// for the stream.  Chunks of horizons, then one block turns them into the
// per-instance offsets.
constexpr int NA_HCHUNK = 960, NA_FCHUNK = 500;
struct HorizonChunk { int n, off; int N[NA_HCHUNK]; };
struct ScheduleChunk { int n, off; double f[NA_FCHUNK]; };

__global__ void na_horizons_kernel(HorizonChunk c, int* N) {
  for (int k = threadIdx.x; k < c.n; k += blockDim.x) N[c.off + k] = c.N[k];
}
__global__ void na_schedule_kernel(ScheduleChunk c, double* f) {
  for (int k = threadIdx.x; k < c.n; k += blockDim.x) f[c.off + k] = c.f[k];
}

// xoff, uoff, soff of every instance (exclusive prefix sums of N + 1, N and
// the exported-state size) by one block of NA_SCAN threads: each thread sums a
// contiguous run of instances, the block scans the run totals, and each thread
// writes its run's offsets.
constexpr int NA_SCAN = 1024;
__global__ void __launch_bounds__(NA_SCAN) na_offsets_kernel(int B, int nx, int nu, int mb, const int* N,
                                                             long long* xoff, long long* uoff, long long* soff) {
  __shared__ long long sx[NA_SCAN], su[NA_SCAN], ss[NA_SCAN];
  const int t = threadIdx.x, per = (B + NA_SCAN - 1) / NA_SCAN;
  const int lo = min(B, t * per), hi = min(B, lo + per);
  long long ax = 0, au = 0, as = 0;
  for (int b = lo; b < hi; ++b) {
    const long long n = N[b];
    ax += n + 1; au += n; as += 6 * (n + 1) * nx + 3 * n * nu + 2 * (n + 1) * mb * 3;
  }
  sx[t] = ax; su[t] = au; ss[t] = as;
  __syncthreads();
  for (int o = 1; o < NA_SCAN; o <<= 1) {   // inclusive Hillis-Steele scan
    long long vx = 0, vu = 0, vs = 0;
    if (t >= o) { vx = sx[t - o]; vu = su[t - o]; vs = ss[t - o]; }
    __syncthreads();
    sx[t] += vx; su[t] += vu; ss[t] += vs;
    __syncthreads();
  }
  long long px = sx[t] - ax, pu = su[t] - au, ps = ss[t] - as;   // exclusive
  for (int b = lo; b < hi; ++b) {
    const long long n = N[b];
    xoff[b] = px; uoff[b] = pu; soff[b] = ps;
    px += n + 1; pu += n; ps += 6 * (n + 1) * nx + 3 * n * nu + 2 * (n + 1) * mb * 3;
  }
}

}  // namespace

extern "C" ucn_status ucn_scp_solve_noalloc(const ucn_problem_desc* d, const double* x0_d, const double* u0_d,
                                            double* x_out_d, double* u_out_d, ucn_scp_stats* stats_d,
                                            int* status_d, void* stream) {
  set_error_message("");
  if (!d || !x0_d || !u0_d || !x_out_d || !u_out_d || !stats_d || !status_d) return nfail(UCN_EINVAL, "null argument");
  if (!model_known(d->model)) return nfail(UCN_EINVAL, "unknown model %d", d->model);
  const int NX = model_nx(d->model), NU = model_nu(d->model);
  const bool obst = model_obstacles(d->model);
  if (d->nx != NX || d->nu != NU) return nfail(UCN_EINVAL, "model %d needs nx=%d nu=%d", d->model, NX, NU);
  if (d->batch < 1) return nfail(UCN_EINVAL, "batch must be >= 1");
  if (d->precision != UCN_PREC_FP64 && d->precision != UCN_PREC_FP32_REFINE) return nfail(UCN_EINVAL, "unknown precision %d", d->precision);
  if (d->vc_weight != 0.0) return nfail(UCN_EINVAL, "virtual control (vc_weight != 0) is not supported");
  if (d->group > 1) return nfail(UCN_EINVAL, "scenario groups run through ucn_scp_solve only");
  if (!d->horizon || !d->dt || !d->model_params || !d->Q_diag || !d->x_ref || !d->R_diag || !d->u_ref ||
      !d->QN_diag || !d->qN || !d->x_lo || !d->x_hi || !d->u_lo || !d->u_hi || !d->x_init || !d->x_target || !d->term_mask)
    return nfail(UCN_EINVAL, "a required descriptor array is NULL");
  const int max_obs = obst ? d->max_obs : 0;
  if (max_obs < 0 || max_obs > 64) return nfail(UCN_EINVAL, "max_obs must be in [0, 64]");
  if (obst && (!d->n_obs || (max_obs > 0 && (!d->obs_c || !d->obs_r))))
    return nfail(UCN_EINVAL, "quadrotor problems need n_obs (and obs_c, obs_r when max_obs > 0)");
  if (!obst && !d->sets) return nfail(UCN_EINVAL, "Mars problems need the sets array");
  if (!(d->rho_eq > 0 && d->rho_dyn > 0 && d->rho_geo > 0)) return nfail(UCN_EINVAL, "penalties must be positive");
  if (d->scp_iters < 1 || d->admm_iters < 1) return nfail(UCN_EINVAL, "iteration counts must be >= 1");
  if (!(d->tr_init > 0 && d->tr_min > 0 && d->tr_max >= d->tr_min)) return nfail(UCN_EINVAL, "bad trust-region bounds");
  const int B = d->batch;
  const int mb = obst ? max_obs : (d->model == UCN_MODEL_MARS14 ? 6 : 3);
  long long ts = 0;
  int Nmax = 0;
  for (int b = 0; b < B; ++b) {
    const long long n = d->horizon[b];
    if (n < 1 || n + 1 > MAX_THREADS) return nfail(UCN_EINVAL, "horizon[%d] = %lld outside [1, %d]", b, n, MAX_THREADS - 1);
    ts += 6 * (n + 1) * NX + 3 * n * NU + 2 * (n + 1) * mb * 3;
    Nmax = std::max(Nmax, (int)n);
  }
  const int K = d->scp_iters;
  const long long oN = 0, oX = up256(4LL * B), oU = oX + up256(8LL * B), oS = oU + up256(8LL * B);
  const long long oF = oS + up256(8LL * B), oState = oF + up256(8LL * K);
  const long long need = oState + 8LL * ts;
  if (need > (long long)UCN_NOALLOC_SCRATCH_BYTES)
    return nfail(UCN_EINVAL, "batch needs %lld bytes of scratch; the no-allocation entry point holds %llu",
                 need, (unsigned long long)UCN_NOALLOC_SCRATCH_BYTES);
  const int tsize = d->precision == UCN_PREC_FP64 ? 8 : 4;
  const int tpn = default_tpn(d->model, Nmax + 1, d->precision);
  const Layout L = make_layout(d->model, Nmax + 1, max_obs, tsize, d->model == UCN_MODEL_MARS7, tpn);
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return nfail(UCN_ECUDA, "no CUDA device"); }
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (L.bytes + (long long)sizeof(InstShared) + 64 > optin)
    return nfail(UCN_EINVAL, "an instance of %d nodes needs %lld bytes of shared memory (device limit %d); "
                 "the no-allocation entry point has no global workspace", Nmax + 1, (long long)L.bytes, optin);
  unsigned char* scr = nullptr;
  cudaError_t e = scratch_address(dev, (void**)&scr);
  if (e != cudaSuccess) return nfail(UCN_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  // tables and schedule in by value (see na_horizons_kernel), offsets on the device
  {
    HorizonChunk hc;
    for (int off = 0; off < B; off += NA_HCHUNK) {
      hc.off = off; hc.n = std::min(NA_HCHUNK, B - off);
      for (int k = 0; k < hc.n; ++k) hc.N[k] = d->horizon[off + k];
      na_horizons_kernel<<<1, 256, 0, st>>>(hc, (int*)(scr + oN));
    }
    ScheduleChunk fc;
    for (int off = 0; off < K; off += NA_FCHUNK) {
      fc.off = off; fc.n = std::min(NA_FCHUNK, K - off);
      for (int k = 0; k < fc.n; ++k) fc.f[k] = rho_factor(d->rho_final, d->rho_geo, K, off + k);
      na_schedule_kernel<<<1, 256, 0, st>>>(fc, (double*)(scr + oF));
    }
    na_offsets_kernel<<<1, NA_SCAN, 0, st>>>(B, NX, NU, mb, (const int*)(scr + oN), (long long*)(scr + oX),
                                            (long long*)(scr + oU), (long long*)(scr + oS));
    if ((e = cudaGetLastError()) != cudaSuccess) return nfail(UCN_ECUDA, "table set-up launch: %s", cudaGetErrorString(e));
  }
  ProblemDev P;
  std::memset(&P, 0, sizeof(P));
  P.model = d->model; P.nx = NX; P.nu = NU; P.batch = B; P.max_obs = max_obs;
  P.N = (const int*)(scr + oN); P.xoff = (const long long*)(scr + oX);
  P.uoff = (const long long*)(scr + oU); P.soff = (const long long*)(scr + oS);
  P.dt = d->dt; P.params = d->model_params; P.Qd = d->Q_diag; P.xref = d->x_ref; P.Rd = d->R_diag; P.uref = d->u_ref;
  P.QNd = d->QN_diag; P.qN = d->qN; P.xlo = d->x_lo; P.xhi = d->x_hi; P.ulo = d->u_lo; P.uhi = d->u_hi;
  P.xinit = d->x_init; P.xtarget = d->x_target; P.tmask = d->term_mask;
  P.nobs = d->n_obs; P.obs_c = d->obs_c; P.obs_r = d->obs_r; P.sets = d->sets;
  P.rho_eq = d->rho_eq; P.rho_dyn = d->rho_dyn; P.rho_geo = d->rho_geo; P.rho_final = d->rho_final;
  P.scp_iters = d->scp_iters; P.admm_iters = d->admm_iters; P.stop = d->stop;
  P.tr_init = d->tr_init; P.tr_min = d->tr_min; P.tr_max = d->tr_max; P.w_d = d->w_d;
  P.defect_tol = d->defect_tol; P.step_tol = d->step_tol;
  P.timeout_ns = (unsigned long long)((d->timeout_s > 0 ? d->timeout_s : 60.0) * 1e9);
  P.state_abs = (double*)(scr + oState);
  P.rho_fac = (const double*)(scr + oF);
  P.ws = nullptr;
  LaunchCfg c;
  c.P = &P; c.L = &L; c.smem = true; c.smem_bytes = L.bytes;
  c.threads = (int)((Nmax + 1 + 31) / 32 * 32); c.blocks = B; c.stream = st; c.group = 1;
  c.nodes = Nmax + 1; c.tpn = tpn;
  auto fn = launchers_for(d->model, d->precision).scp;
  e = fn(c, x0_d, u0_d, x_out_d, u_out_d, stats_d, status_d);
  if (e != cudaSuccess) return nfail(UCN_ECUDA, "scp launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}
