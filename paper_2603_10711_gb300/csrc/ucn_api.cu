// C-ABI implementation: descriptor validation, device copies, workspace
// sizing and kernel dispatch.  See include/ucn.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ucn_internal.h"
#include "ucn_kernels.cuh"
#include "ucn_lanes.cuh"
#include "ucn_pair.cuh"

using namespace ucn;

namespace {

thread_local char g_err[512] = "";

ucn_status fail(ucn_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

}  // namespace

namespace ucn {

void set_error_message(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

int fault_alloc_at() {
  const char* e = std::getenv("UCN_FAULT_ALLOC");
  return e ? std::atoi(e) : 0;
}

bool tpn_allowed(int tpn, int model, int nodes, int precision, bool smem) {
  if (tpn == 1) return true;
  if (tpn == 4) return model == UCN_MODEL_QUAD12 && 4 * nodes <= LANES_MAX_THREADS;
  if (tpn == 2)
    return model == UCN_MODEL_MARS7 && precision == UCN_PREC_FP32_REFINE && smem &&
           (2 * nodes + 31) / 32 * 32 <= PAIR_MAX_THREADS;
  return false;
}

int default_tpn(int model, int nodes, int precision) {
  if (tpn_allowed(4, model, nodes, precision, true)) return 4;
  return 1;
}

double rho_factor(double rho_final, double rho_geo, int K, int k) {
  return (rho_final > 0.0 && K > 1) ? std::pow(rho_final / rho_geo, (double)k / (double)(K - 1)) : 1.0;
}

std::vector<double> rho_schedule(double rho_final, double rho_geo, int K) {
  std::vector<double> fac(std::max(K, 1), 1.0);
  for (int k = 0; k < (int)fac.size(); ++k) fac[k] = rho_factor(rho_final, rho_geo, K, k);
  return fac;
}

Layout make_layout(int model, int nodes, int max_obs, int tsize, bool reg_mats, int tpn) {
  const bool quad = model_obstacles(model);
  const int NX = model_nx(model), NU = model_nu(model), NN = NX + NU;
  const int fixed = model == UCN_MODEL_QUAD12 ? Rec<Quad12>::END                 // fixed part of a node record
                    : model == UCN_MODEL_QUAT13 ? Rec<Quat13>::END
                    : model == UCN_MODEL_MARS14 ? Rec<Mars14>::END : Rec<Mars7>::END;
  const int dfixed = model == UCN_MODEL_QUAD12 ? Rec<Quad12>::DEND
                     : model == UCN_MODEL_QUAT13 ? Rec<Quat13>::DEND
                     : model == UCN_MODEL_MARS14 ? Rec<Mars14>::DEND : Rec<Mars7>::DEND;
  Layout L;
  std::memset(&L, 0, sizeof(L));
  const int mo = std::max(max_obs, 1);
  const bool m14 = model == UCN_MODEL_MARS14;
  L.MS = quad ? mo : (m14 ? M14::MS : 7);
  L.MD = quad ? (tsize == 4 ? 5 : 4) * mo : (m14 ? M14::MD : 10);   // ObsStride; Mars: nbar, bound, position, thrust (+ qyz, rates)
  L.MB = quad ? max_obs : (m14 ? 6 : 3);
  L.oS = fixed;
  L.oNus = fixed + L.MS;
  L.oMd = fixed + 2 * L.MS;
  int nt = fixed + 2 * L.MS + L.MD;
  if (reg_mats) {
    L.oA = L.oB = L.oH = -1;
  } else {
    const bool pad = model == UCN_MODEL_QUAD12 && tsize == 4;   // MatStride: the FP32 lane layout
    L.oA = nt; L.oB = L.oA + NX * (pad ? (NX | 1) : NX); L.oH = L.oB + NX * (pad ? (NU | 1) : NU);
    nt = L.oH + NN * (NN + 1) / 2;
  }
  L.S = nodes;
  // Record stride: odd for one thread per node (consecutive nodes fall in
  // distinct banks); 4 mod 32 for the lane kernel, whose warps read 8 nodes x
  // 4 consecutive row elements, and twice an odd number for the pair kernel,
  // whose warps read 16 nodes x 2 consecutive row elements -- 32 distinct banks.
  L.NS = tpn == 4 ? nt + ((4 - nt) % 32 + 32) % 32 : tpn == 2 ? nt + ((2 - nt) % 4 + 4) % 4 : (nt | 1);
  L.DS = dfixed | 1;
  L.tbytes = round_up((long long)nodes * L.NS * tsize, 16);
  L.bytes = round_up(L.tbytes + (long long)nodes * L.DS * 8, 16);
  // FP32 path: the instance's constants in double-float (CB block) follow
  L.oC = -1;
  if (tsize == 4) {
    const int cb = model == UCN_MODEL_QUAD12 ? CB<Quad12>::END
                   : model == UCN_MODEL_QUAT13 ? CB<Quat13>::END
                   : model == UCN_MODEL_MARS14 ? CB<Mars14>::END : CB<Mars7>::END;
    L.oC = L.bytes;
    L.bytes = round_up(L.bytes + 8LL * cb, 16);
  }
  // pair kernel: one H^-1 record per thread (two per node)
  L.oPH = -1;
  if (tpn == 2) {
    L.oPH = L.bytes;
    L.bytes += (long long)((2 * nodes + 31) / 32 * 32) * PAIR_HREC * 4;
  }
  return L;
}

}  // namespace ucn

struct ucn_problem {
  int model, nx, nu, batch, max_obs, Nmax, precision;
  long long total_x, total_u, state_size;
  std::vector<void*> allocs;
  ProblemDev dev;
  Layout L;
  bool smem;
  long long smem_bytes;
  int threads;
  int* node_inst;
  int* order_d;
  int group, gcsize;     // scenarios per group, CTAs per thread-block cluster
  int tpn;               // threads per node of the fused solve
  int last_launches = 0; // kernel launches of the last fused solve
  int optin;             // shared memory per CTA the device allows
  unsigned char* warm_ones;   // batch flags, all 1: every instance starts from the given state
};

namespace {

template <class V>
ucn_status dev_copy(ucn_problem* p, int& nalloc, int fault_at, const V* host, size_t n, V** out) {
  ++nalloc;
  if (fault_at > 0 && nalloc == fault_at) return fail(UCN_ENOMEM, "injected allocation failure (UCN_FAULT_ALLOC=%d)", fault_at);
  void* d = nullptr;
  const size_t bytes = std::max<size_t>(n * sizeof(V), 16);
  if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return fail(UCN_ENOMEM, "cudaMalloc of %zu bytes failed", bytes); }
  p->allocs.push_back(d);
  if (host && n) {
    const cudaError_t e = cudaMemcpy(d, host, n * sizeof(V), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(UCN_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  } else {
    cudaMemset(d, 0, bytes);
  }
  *out = (V*)d;
  return UCN_OK;
}

cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

}  // namespace

namespace {

// Receding-horizon step (Sec. IV-A): the plant -- the model of the group's
// first instance -- takes the applied first control for one step from the
// current initial state; every instance's next guess is its solution shifted
// by one node (last node and control repeated) starting at the new state.
template <class M>
__global__ void mpc_shift_kernel(ProblemDev P, const double* x, const double* u, double* xg, double* ug) {
  constexpr int NX = M::NX, NU = M::NU;
  const int b = blockIdx.x, N = P.N[b];
  const int lead = P.group > 1 ? b - b % P.group : b;
  const long long xo = P.xoff[b], uo = P.uoff[b];
  __shared__ double x0n[NX];
  if (threadIdx.x == 0) {
    double xi[NX], ui[NU];
    for (int j = 0; j < NX; ++j) xi[j] = P.xinit[lead * NX + j];
    for (int j = 0; j < NU; ++j) ui[j] = u[P.uoff[lead] * NU + j];
    rk4<M, double>(P.params + lead * 8, P.dt[lead], xi, ui, x0n);
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
    const long long src = xo + (i < N ? i + 1 : N);
    for (int j = 0; j < NX; ++j) xg[(xo + i) * NX + j] = i == 0 ? x0n[j] : x[src * NX + j];
    if (i < N) {
      const long long su = uo + (i + 1 < N ? i + 1 : N - 1);
      for (int j = 0; j < NU; ++j) ug[(uo + i) * NU + j] = u[su * NU + j];
    }
  }
}

// The problem's initial states <- node 0 of the shifted guesses.
__global__ void mpc_set_init_kernel(ProblemDev P, double* xinit, const double* xg) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.batch * P.nx) return;
  const int b = k / P.nx, j = k % P.nx;
  xinit[k] = xg[P.xoff[b] * P.nx + j];
}

}  // namespace

extern "C" {

const char* ucn_last_error(void) { return g_err; }

void ucn_problem_destroy(ucn_problem* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  for (void* a : p->allocs) cudaFree(a);
  delete p;
}

ucn_status ucn_problem_create(const ucn_problem_desc* d, ucn_problem** out) {
  g_err[0] = 0;
  if (!d || !out) return fail(UCN_EINVAL, "null descriptor or output pointer");
  *out = nullptr;
  if (!model_known(d->model)) return fail(UCN_EINVAL, "unknown model %d", d->model);
  const int NX = model_nx(d->model), NU = model_nu(d->model);
  const bool obst = model_obstacles(d->model);
  if (d->nx != NX || d->nu != NU) return fail(UCN_EINVAL, "model %d needs nx=%d nu=%d (got %d, %d)", d->model, NX, NU, d->nx, d->nu);
  if (d->batch < 1) return fail(UCN_EINVAL, "batch must be >= 1 (got %d)", d->batch);
  if (d->precision != UCN_PREC_FP64 && d->precision != UCN_PREC_FP32_REFINE) return fail(UCN_EINVAL, "unknown precision %d", d->precision);
  if (d->vc_weight != 0.0) return fail(UCN_EINVAL, "virtual control (vc_weight != 0) is not supported");
  if (!d->horizon || !d->dt || !d->model_params || !d->Q_diag || !d->x_ref || !d->R_diag || !d->u_ref ||
      !d->QN_diag || !d->qN || !d->x_lo || !d->x_hi || !d->u_lo || !d->u_hi || !d->x_init || !d->x_target ||
      !d->term_mask)
    return fail(UCN_EINVAL, "a required descriptor array is NULL");
  if (obst && d->max_obs > 0 && (!d->n_obs || !d->obs_c || !d->obs_r))
    return fail(UCN_EINVAL, "obstacle arrays are NULL with max_obs > 0");
  if (!obst && !d->sets) return fail(UCN_EINVAL, "Mars problems need the sets array");
  if (d->max_obs < 0 || d->max_obs > 64) return fail(UCN_EINVAL, "max_obs must be in [0, 64]");
  if (!(d->rho_eq > 0 && d->rho_dyn > 0 && d->rho_geo > 0)) return fail(UCN_EINVAL, "penalties must be positive");
  if (d->scp_iters < 1 || d->admm_iters < 1) return fail(UCN_EINVAL, "iteration counts must be >= 1");
  if (!(d->tr_init > 0 && d->tr_min > 0 && d->tr_max >= d->tr_min)) return fail(UCN_EINVAL, "bad trust-region bounds");
  const int group = d->group > 1 ? d->group : 1;
  if (d->group < 0 || group > UCN_MAX_GROUP) return fail(UCN_EINVAL, "group must be in [0, %d] (got %d)", UCN_MAX_GROUP, d->group);
  if (group > 1 && d->model != UCN_MODEL_QUAD12) return fail(UCN_EINVAL, "scenario groups need the quadrotor model");
  if (group > 1 && d->batch % group) return fail(UCN_EINVAL, "batch %d is not a multiple of group %d", d->batch, group);
  int Nmax = 0;
  for (int b = 0; b < d->batch; ++b) {
    const int N = d->horizon[b];
    if (N < 1 || N + 1 > MAX_THREADS) return fail(UCN_EINVAL, "horizon[%d] = %d outside [1, %d]", b, N, MAX_THREADS - 1);
    if (!(d->dt[b] > 0)) return fail(UCN_EINVAL, "dt[%d] must be positive", b);
    if (obst && d->max_obs > 0 && (d->n_obs[b] < 0 || d->n_obs[b] > d->max_obs))
      return fail(UCN_EINVAL, "n_obs[%d] = %d outside [0, max_obs]", b, d->n_obs[b]);
    Nmax = std::max(Nmax, N);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return fail(UCN_ECUDA, "no CUDA device"); }
  ucn_problem* p = new ucn_problem();
  p->model = d->model; p->nx = NX; p->nu = NU; p->batch = d->batch; p->max_obs = obst ? d->max_obs : 0;
  p->Nmax = Nmax; p->precision = d->precision; p->group = group;
  p->tpn = default_tpn(d->model, Nmax + 1, d->precision);
  const int B = d->batch;
  std::vector<long long> xoff(B), uoff(B), soff(B);
  std::vector<int> node_inst;
  const int mb = obst ? p->max_obs : (d->model == UCN_MODEL_MARS14 ? 6 : 3);
  long long tx = 0, tu = 0, ts = 0;
  for (int b = 0; b < B; ++b) {
    const long long N = d->horizon[b];
    xoff[b] = tx; uoff[b] = tu; soff[b] = ts;
    tx += N + 1; tu += N;
    ts += 6 * (N + 1) * NX + 3 * N * NU + 2 * (N + 1) * mb * 3;
    for (long long i = 0; i < N; ++i) node_inst.push_back(b);
  }
  p->total_x = tx; p->total_u = tu; p->state_size = ts;
  const int fa = fault_alloc_at();
  int na = 0;
  ucn_status s = UCN_OK;
  ProblemDev& P = p->dev;
  std::memset(&P, 0, sizeof(P));
  P.model = d->model; P.nx = NX; P.nu = NU; P.batch = B; P.max_obs = p->max_obs;
  std::vector<double> zeros_obs(1, 0.0);
  std::vector<int> zeros_nobs(B, 0);
  std::vector<double> zeros_sets((size_t)B * UCN_SET_PARAMS, 0.0);
#define COPY(dst, src, n)                                                                  \
  if (s == UCN_OK) { s = dev_copy(p, na, fa, src, (size_t)(n), &dst); }
  int* Ndev = nullptr; long long *xo = nullptr, *uo = nullptr, *so = nullptr;
  double *dtd, *prm, *Qd, *xr, *Rd, *ur, *QNd, *qN, *xlo, *xhi, *ulo, *uhi, *xi, *xt, *oc, *orr, *sets;
  unsigned char* tm; int* nobs;
  COPY(Ndev, d->horizon, B); COPY(xo, xoff.data(), B); COPY(uo, uoff.data(), B); COPY(so, soff.data(), B);
  COPY(dtd, d->dt, B); COPY(prm, d->model_params, (size_t)B * 8);
  COPY(Qd, d->Q_diag, (size_t)B * NX); COPY(xr, d->x_ref, (size_t)B * NX);
  COPY(Rd, d->R_diag, (size_t)B * NU); COPY(ur, d->u_ref, (size_t)B * NU);
  COPY(QNd, d->QN_diag, (size_t)B * NX); COPY(qN, d->qN, (size_t)B * NX);
  COPY(xlo, d->x_lo, (size_t)B * NX); COPY(xhi, d->x_hi, (size_t)B * NX);
  COPY(ulo, d->u_lo, (size_t)B * NU); COPY(uhi, d->u_hi, (size_t)B * NU);
  COPY(xi, d->x_init, (size_t)B * NX); COPY(xt, d->x_target, (size_t)B * NX);
  COPY(tm, d->term_mask, (size_t)B * NX);
  if (p->max_obs > 0) {
    COPY(nobs, d->n_obs, B); COPY(oc, d->obs_c, (size_t)B * p->max_obs * 3); COPY(orr, d->obs_r, (size_t)B * p->max_obs);
  } else {
    COPY(nobs, zeros_nobs.data(), B); COPY(oc, zeros_obs.data(), 1); COPY(orr, zeros_obs.data(), 1);
  }
  COPY(sets, d->sets ? d->sets : zeros_sets.data(), (size_t)B * UCN_SET_PARAMS);
  int* ni = nullptr;
  COPY(ni, node_inst.empty() ? zeros_nobs.data() : node_inst.data(), std::max<size_t>(node_inst.size(), 1));
  // default CTA order of the fused solve: largest estimated work first
  // (nodes x (1 + obstacles / 8)), ties by index -- a longest-processing-time
  // schedule for uneven batches; results do not depend on it
  std::vector<int> order(B);
  for (int b = 0; b < B; ++b) order[b] = b;
  {
    std::vector<double> w(B);
    for (int b = 0; b < B; ++b)
      w[b] = (d->horizon[b] + 1.0) * (1.0 + ((obst && d->max_obs > 0) ? d->n_obs[b] / 8.0 : 0.0));
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return w[x] > w[y]; });
  }
  int* ord = nullptr;
  COPY(ord, order.data(), B);
  const std::vector<double> fac = rho_schedule(d->rho_final, d->rho_geo, d->scp_iters);
  double* facd = nullptr;
  COPY(facd, fac.data(), fac.size());
  double* sabs = nullptr;
  COPY(sabs, (const double*)nullptr, (size_t)ts);
  const std::vector<unsigned char> ones(B, 1);
  unsigned char* wones = nullptr;
  COPY(wones, ones.data(), B);
#undef COPY
  if (s != UCN_OK) { ucn_problem_destroy(p); return s; }
  P.N = Ndev; P.xoff = xo; P.uoff = uo; P.soff = so; P.dt = dtd; P.params = prm;
  P.Qd = Qd; P.xref = xr; P.Rd = Rd; P.uref = ur; P.QNd = QNd; P.qN = qN;
  P.xlo = xlo; P.xhi = xhi; P.ulo = ulo; P.uhi = uhi; P.xinit = xi; P.xtarget = xt; P.tmask = tm;
  P.nobs = nobs; P.obs_c = oc; P.obs_r = orr; P.sets = sets;
  P.rho_eq = d->rho_eq; P.rho_dyn = d->rho_dyn; P.rho_geo = d->rho_geo; P.rho_final = d->rho_final;
  P.scp_iters = d->scp_iters; P.admm_iters = d->admm_iters; P.stop = d->stop;
  P.tr_init = d->tr_init; P.tr_min = d->tr_min; P.tr_max = d->tr_max; P.w_d = d->w_d;
  P.defect_tol = d->defect_tol; P.step_tol = d->step_tol;
  P.timeout_ns = (unsigned long long)((d->timeout_s > 0 ? d->timeout_s : 60.0) * 1e9);
  P.state_abs = sabs;
  P.order = ord;
  p->warm_ones = wones;
  P.rho_fac = facd;
  P.group = group;
  // a group is gclusters thread-block clusters of gcsize CTAs: a group of up to
  // 16 scenarios is one cluster (its exchange stays in distributed shared
  // memory: 16 scenarios 1.7x faster than clusters of 2); a larger group runs
  // as clusters of 2 CTAs (1 if the group is odd) that combine through global
  // memory -- measured on GB300 with 64 scenarios per problem, 20% faster than
  // clusters of 16, whose 16-CTA co-scheduling leaves SMs idle
  const int gcsize = group <= 16 ? group : (group % 2 == 0 ? 2 : 1);
  p->gcsize = gcsize;
  P.gclusters = group / gcsize;
  // bound on a wait for another scenario (the group runs in lockstep, so waits
  // are short; the bound only guarantees that the kernel ends)
  P.gwait_ns = 10ull * 1000000000ull;
  p->node_inst = ni;
  p->order_d = ord;
  // per-node storage: shared memory when one instance fits (small models then keep
  // their matrices in registers), else a structure-of-arrays slice of global memory
  const int tsize = d->precision == UCN_PREC_FP64 ? 8 : 4;
  const bool small = d->model == UCN_MODEL_MARS7;   // SmallModel<Mars7> (registers hold A, B, H^-1)
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const long long static_sh = (long long)sizeof(InstShared) + (group > 1 ? (long long)sizeof(GroupShared) : 0) + 64;
  p->L = make_layout(d->model, Nmax + 1, p->max_obs, tsize, small, p->tpn);
  p->smem = p->L.bytes + static_sh <= optin;
  if (!p->smem) {
    if (!tpn_allowed(p->tpn, d->model, Nmax + 1, d->precision, false)) p->tpn = 1;
    p->L = make_layout(d->model, Nmax + 1, p->max_obs, tsize, false, p->tpn);
  }
  p->optin = optin;
  p->threads = (int)round_up(Nmax + 1, 32);
  p->smem_bytes = p->smem ? p->L.bytes : 0;
  if (group > 1 && !p->smem) {
    ucn_problem_destroy(p);
    return fail(UCN_EINVAL, "scenario groups need node records in shared memory (horizon or obstacle count too large)");
  }
  if (group > 1) {
    // exchange slots and counters of the scenarios
    const size_t nc = (size_t)B;
    const bool injected = fa > 0 && (na + 1 == fa || na + 2 == fa);
    na += 2;
    void* gx = nullptr;
    void* gf = nullptr;
    if (injected || cudaMalloc(&gx, nc * 2 * 16 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      ucn_problem_destroy(p);
      return fail(UCN_ENOMEM, "group exchange slots");
    }
    p->allocs.push_back(gx);
    if (cudaMalloc(&gf, nc * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      ucn_problem_destroy(p);
      return fail(UCN_ENOMEM, "group exchange counters");
    }
    p->allocs.push_back(gf);
    P.gx = (double*)gx;
    P.gflag = (unsigned*)gf;
  }
  P.ws = nullptr;
  if (!p->smem) {
    char* ws = nullptr;
    ++na;
    if (fa > 0 && na == fa) { ucn_problem_destroy(p); return fail(UCN_ENOMEM, "injected allocation failure (UCN_FAULT_ALLOC=%d)", fa); }
    if (cudaMalloc(&ws, (size_t)(p->L.bytes * B)) != cudaSuccess) {
      cudaGetLastError();
      ucn_problem_destroy(p);
      return fail(UCN_ENOMEM, "workspace of %lld bytes", (long long)(p->L.bytes * B));
    }
    p->allocs.push_back(ws);
    P.ws = ws;
  }
  *out = p;
  return UCN_OK;
}

ucn_status ucn_problem_set_order(ucn_problem* p, const int* order) {
  g_err[0] = 0;
  if (!p) return fail(UCN_EINVAL, "null problem");
  if (p->group > 1) return fail(UCN_EINVAL, "grouped problems run their clusters in instance order");
  std::vector<int> o(p->batch);
  if (order) {
    std::vector<char> seen(p->batch, 0);
    for (int b = 0; b < p->batch; ++b) {
      if (order[b] < 0 || order[b] >= p->batch || seen[order[b]]) return fail(UCN_EINVAL, "order is not a permutation of 0..batch-1");
      seen[order[b]] = 1;
      o[b] = order[b];
    }
  } else {
    for (int b = 0; b < p->batch; ++b) o[b] = b;
  }
  const cudaError_t e = cudaMemcpy(p->order_d, o.data(), sizeof(int) * p->batch, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(UCN_ECUDA, "order copy: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_problem_set_lanes(ucn_problem* p, int lanes_per_node) {
  g_err[0] = 0;
  if (!p) return fail(UCN_EINVAL, "null problem");
  if (!tpn_allowed(lanes_per_node, p->model, p->Nmax + 1, p->precision, p->smem))
    return fail(UCN_EINVAL, "%d threads per node: 1; 2 for 3-DOF Mars problems of at most %d nodes on the FP32 path; "
                "4 for quadrotor problems of at most %d nodes", lanes_per_node, PAIR_MAX_THREADS / 2,
                LANES_MAX_THREADS / 4);
  if (p->smem && lanes_per_node != p->tpn) {
    // the record stride follows the threads per node (bank-conflict-free reads)
    const Layout L = make_layout(p->model, p->Nmax + 1, p->max_obs, p->precision == UCN_PREC_FP64 ? 8 : 4,
                                 p->model == UCN_MODEL_MARS7, lanes_per_node);
    const long long static_sh = (long long)sizeof(InstShared) + (p->group > 1 ? (long long)sizeof(GroupShared) : 0) + 64;
    if (L.bytes + static_sh > p->optin) return fail(UCN_EINVAL, "the %d-thread layout does not fit in shared memory", lanes_per_node);
    p->L = L;
    p->smem_bytes = L.bytes;
  }
  p->tpn = lanes_per_node;
  return UCN_OK;
}

int ucn_problem_lanes(const ucn_problem* p) { return p ? p->tpn : -1; }

int ucn_problem_last_launches(const ucn_problem* p) { return p ? p->last_launches : -1; }

long long ucn_total_x(const ucn_problem* p) { return p ? p->total_x : -1; }
long long ucn_total_u(const ucn_problem* p) { return p ? p->total_u : -1; }
long long ucn_state_size(const ucn_problem* p) { return p ? p->state_size : -1; }

static LaunchCfg cfg_of(ucn_problem* p, void* stream) {
  LaunchCfg c;
  c.P = &p->dev; c.L = &p->L; c.smem = p->smem; c.smem_bytes = p->smem_bytes;
  c.threads = p->threads; c.blocks = p->batch; c.stream = as_stream(stream); c.group = p->gcsize;
  c.nodes = p->Nmax + 1; c.tpn = p->tpn;
  c.launched = &p->last_launches;
  p->last_launches = 1;   // one launch unless the launcher splits the batch
  return c;
}

ucn_status ucn_linearize(ucn_problem* p, const double* xbar_d, const double* ubar_d, double* A_d, double* B_d,
                         double* d_d, void* stream) {
  g_err[0] = 0;
  if (!p || !xbar_d || !ubar_d || !A_d || !B_d || !d_d) return fail(UCN_EINVAL, "null argument");
  auto fn = launchers_for(p->model, p->precision).linearize;
  const cudaError_t e = fn(&p->dev, p->node_inst, p->total_u, xbar_d, ubar_d, A_d, B_d, d_d, as_stream(stream));
  if (e != cudaSuccess) return fail(UCN_ECUDA, "linearize launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_admm_solve(ucn_problem* p, const double* xbar_d, const double* ubar_d, const double* A_d,
                          const double* B_d, const double* d_d, const double* radius_d, int iters, int warm,
                          double* xhat_d, double* uhat_d, double* res_d, int* status_d, void* stream) {
  g_err[0] = 0;
  if (!p || !xbar_d || !ubar_d || !A_d || !B_d || !d_d || !radius_d || !xhat_d || !uhat_d || !res_d || !status_d)
    return fail(UCN_EINVAL, "null argument");
  if (iters < 1) return fail(UCN_EINVAL, "iters must be >= 1");
  if (p->group > 1) return fail(UCN_EINVAL, "the scenario consensus runs inside ucn_scp_solve only");
  const LaunchCfg c = cfg_of(p, stream);
  auto fn = launchers_for(p->model, p->precision).admm;
  const cudaError_t e = fn(c, xbar_d, ubar_d, A_d, B_d, d_d, radius_d, iters, warm ? 1 : 0, xhat_d, uhat_d, res_d, status_d);
  if (e != cudaSuccess) return fail(UCN_ECUDA, "admm launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_state_export(ucn_problem* p, double* state_d, void* stream) {
  g_err[0] = 0;
  if (!p || !state_d) return fail(UCN_EINVAL, "null argument");
  const cudaError_t e = cudaMemcpyAsync(state_d, p->dev.state_abs, (size_t)p->state_size * sizeof(double),
                                        cudaMemcpyDeviceToDevice, as_stream(stream));
  if (e != cudaSuccess) return fail(UCN_ECUDA, "state export: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_scp_solve(ucn_problem* p, const double* x0_d, const double* u0_d, double* x_out_d, double* u_out_d,
                         ucn_scp_stats* stats_d, int* status_d, void* stream) {
  g_err[0] = 0;
  if (!p || !x0_d || !u0_d || !x_out_d || !u_out_d || !stats_d || !status_d) return fail(UCN_EINVAL, "null argument");
  const LaunchCfg c = cfg_of(p, stream);
  if (p->group > 1) {
    {
      const cudaError_t e = cudaMemsetAsync(p->dev.gflag, 0, sizeof(unsigned) * p->batch, c.stream);
      if (e != cudaSuccess) return fail(UCN_ECUDA, "group counters: %s", cudaGetErrorString(e));
    }
    const cudaError_t e = (p->precision == UCN_PREC_FP64 ? quad64_scp_group : quad32_scp_group)(
        c, x0_d, u0_d, x_out_d, u_out_d, stats_d, status_d);
    if (e == cudaErrorInvalidClusterSize)
      return fail(UCN_EINVAL, "%d clusters of %d CTAs (%d threads, %lld B shared memory each) cannot be resident together",
                  p->dev.gclusters, p->gcsize, p->threads, p->smem_bytes);
    if (e != cudaSuccess) return fail(UCN_ECUDA, "scp group launch: %s", cudaGetErrorString(e));
    return UCN_OK;
  }
  auto fn = launchers_for(p->model, p->precision).scp;
  const cudaError_t e = fn(c, x0_d, u0_d, x_out_d, u_out_d, stats_d, status_d);
  if (e != cudaSuccess) return fail(UCN_ECUDA, "scp launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_scp_solve_warm(ucn_problem* p, const double* x0_d, const double* u0_d, const double* state_d,
                              double* x_out_d, double* u_out_d, ucn_scp_stats* stats_d, int* status_d, void* stream) {
  g_err[0] = 0;
  if (!p || !x0_d || !u0_d || !state_d || !x_out_d || !u_out_d || !stats_d || !status_d)
    return fail(UCN_EINVAL, "null argument");
  if (p->group > 1) return fail(UCN_EINVAL, "scenario groups start cold (warm-start them through their guesses)");
  if (state_d != p->dev.state_abs) {
    const cudaError_t e = cudaMemcpyAsync(p->dev.state_abs, state_d, (size_t)p->state_size * sizeof(double),
                                          cudaMemcpyDeviceToDevice, as_stream(stream));
    if (e != cudaSuccess) return fail(UCN_ECUDA, "state copy: %s", cudaGetErrorString(e));
  }
  ProblemDev Pw = p->dev;
  Pw.warm = p->warm_ones;
  LaunchCfg c = cfg_of(p, stream);
  c.P = &Pw;
  auto fn = launchers_for(p->model, p->precision).scp;
  const cudaError_t e = fn(c, x0_d, u0_d, x_out_d, u_out_d, stats_d, status_d);
  if (e != cudaSuccess) return fail(UCN_ECUDA, "scp launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_mpc_shift(ucn_problem* p, const double* x_d, const double* u_d, double* xg_d, double* ug_d,
                         void* stream) {
  g_err[0] = 0;
  if (!p || !x_d || !u_d || !xg_d || !ug_d) return fail(UCN_EINVAL, "null argument");
  if ((const double*)xg_d == x_d || (const double*)ug_d == u_d) return fail(UCN_EINVAL, "the shifted guesses may not alias the solution");
  const cudaStream_t st = as_stream(stream);
  if (p->model == UCN_MODEL_QUAD12) mpc_shift_kernel<Quad12><<<p->batch, 64, 0, st>>>(p->dev, x_d, u_d, xg_d, ug_d);
  else if (p->model == UCN_MODEL_QUAT13) mpc_shift_kernel<Quat13><<<p->batch, 64, 0, st>>>(p->dev, x_d, u_d, xg_d, ug_d);
  else if (p->model == UCN_MODEL_MARS14) mpc_shift_kernel<Mars14><<<p->batch, 64, 0, st>>>(p->dev, x_d, u_d, xg_d, ug_d);
  else mpc_shift_kernel<Mars7><<<p->batch, 64, 0, st>>>(p->dev, x_d, u_d, xg_d, ug_d);
  const int nx = p->nx;
  mpc_set_init_kernel<<<(p->batch * nx + 127) / 128, 128, 0, st>>>(p->dev, const_cast<double*>(p->dev.xinit), xg_d);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(UCN_ECUDA, "mpc shift launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}

}  // extern "C"
