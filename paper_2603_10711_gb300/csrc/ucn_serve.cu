// Serving: continuous batching of SCP solves over a preallocated slot pool.
//
// All device memory is allocated once by ucn_serve_create, for `max_slots`
// instances of up to `max_horizon` nodes (problem data, guesses, outputs,
// exported state, workspace) plus a ring of kept trajectories for warm
// starts.  Requests are admitted into free slots while their HBM footprint
// fits the budget; every pump launches the fused SCP kernel over the slots
// admitted since the last pump, on the next free lane (a CUDA stream), while
// earlier launches keep running on the other lanes.  A finished request is
// collected by a non-blocking poll, which frees its slot for the next arrival.
// Each instance's solve is independent of the others in its launch (one CTA
// per instance, same CTA size and layout for every slot), so a result does
// not depend on what it was batched with.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ucn_internal.h"
#include "ucn_kernels.cuh"

using namespace ucn;

namespace {

ucn_status sfail(ucn_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_error_message(buf);
  return s;
}

enum { SLOT_FREE = 0, SLOT_ADMITTED = 1, SLOT_RUNNING = 2 };

}  // namespace

struct ucn_server {
  ucn_serve_config cfg;
  int nx, nu, S, Nmax, max_obs, lanes;
  long long state_per_slot, budget, used;
  ProblemDev P;
  Layout L;
  bool smem;
  long long smem_bytes;
  int threads;
  int tpn;               // threads per node of the fused solve
  std::vector<void*> dev_allocs, host_allocs;
  // pinned host mirrors of the per-slot problem arrays (same layout as on the device)
  int *hN, *hnobs;
  double *hdt, *hprm, *hQd, *hxr, *hRd, *hur, *hQNd, *hqN, *hxlo, *hxhi, *hulo, *huhi, *hxi, *hxt, *hoc, *hor, *hsets;
  unsigned char* htm;
  double *hxg, *hug;
  // device
  int *dN, *dnobs;
  double *ddt, *dprm, *dQd, *dxr, *dRd, *dur, *dQNd, *dqN, *dxlo, *dxhi, *dulo, *duhi, *dxi, *dxt, *doc, *dor, *dsets;
  unsigned char* dtm;
  double *x0, *u0, *xo, *uo;
  ucn_scp_stats* stats;
  int* status;
  // slots
  std::vector<int> slot_state, slot_lane, slot_warm_ring;
  std::vector<unsigned long long> slot_ticket;
  std::vector<long long> slot_bytes;
  std::map<unsigned long long, int> ticket_slot;
  unsigned long long next_ticket;
  // lanes
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<int*> order_d;
  std::vector<int*> order_h;
  std::vector<int> lane_busy;
  // kept trajectories (warm starts)
  int R, ring_next;
  double *ring_x, *ring_u;
  std::vector<unsigned long long> ring_ticket;
  std::vector<int> ring_N;
  std::mutex mu;
};

namespace {

template <class V>
bool dalloc(ucn_server* s, V** out, size_t n) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n * sizeof(V), 16)) != cudaSuccess) { cudaGetLastError(); return false; }
  cudaMemset(p, 0, std::max<size_t>(n * sizeof(V), 16));
  s->dev_allocs.push_back(p);
  *out = (V*)p;
  return true;
}

template <class V>
bool halloc(ucn_server* s, V** out, size_t n) {
  void* p = nullptr;
  if (cudaMallocHost(&p, std::max<size_t>(n * sizeof(V), 16)) != cudaSuccess) { cudaGetLastError(); return false; }
  std::memset(p, 0, std::max<size_t>(n * sizeof(V), 16));
  s->host_allocs.push_back(p);
  *out = (V*)p;
  return true;
}

long long footprint(const ucn_server* s, int N) {
  const long long nodes = N + 1;
  long long b = nodes * (long long)(s->nx + s->nu) * 8 * 2;                       // guess + output
  const int mb = model_obstacles(s->cfg.model) ? s->max_obs : (s->cfg.model == UCN_MODEL_MARS14 ? 6 : 3);
  b += 8LL * (6 * nodes * s->nx + 3LL * N * s->nu + 2 * nodes * mb * 3);          // exported state
  if (!s->smem) b += (long long)s->L.bytes * nodes / (s->Nmax + 1);               // global workspace share
  return b;
}

}  // namespace

extern "C" {

void ucn_serve_destroy(ucn_server* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : s->done) cudaEventDestroy(e);
  for (void* p : s->dev_allocs) cudaFree(p);
  for (void* p : s->host_allocs) cudaFreeHost(p);
  delete s;
}

ucn_status ucn_serve_create(const ucn_serve_config* c, ucn_server** out) {
  set_error_message("");
  if (!c || !out) return sfail(UCN_EINVAL, "null argument");
  *out = nullptr;
  if (!model_known(c->model)) return sfail(UCN_EINVAL, "unknown model %d", c->model);
  if (c->precision != UCN_PREC_FP64 && c->precision != UCN_PREC_FP32_REFINE) return sfail(UCN_EINVAL, "unknown precision");
  if (c->max_slots < 1 || c->max_horizon < 1 || c->max_horizon + 1 > MAX_THREADS) return sfail(UCN_EINVAL, "bad slot count or horizon");
  if (c->max_obs < 0 || c->max_obs > 64) return sfail(UCN_EINVAL, "max_obs must be in [0, 64]");
  if (c->lanes < 1 || c->lanes > 16) return sfail(UCN_EINVAL, "lanes must be in [1, 16]");
  if (!(c->rho_eq > 0 && c->rho_dyn > 0 && c->rho_geo > 0) || c->scp_iters < 1 || c->admm_iters < 1)
    return sfail(UCN_EINVAL, "bad penalties or iteration counts");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return sfail(UCN_ECUDA, "no CUDA device"); }
  ucn_server* s = new ucn_server();
  s->cfg = *c;
  const bool quad = model_obstacles(c->model);
  s->nx = model_nx(c->model); s->nu = model_nu(c->model);
  s->S = c->max_slots; s->Nmax = c->max_horizon; s->max_obs = quad ? c->max_obs : 0; s->lanes = c->lanes;
  const int S = s->S, NX = s->nx, NU = s->nu, MO = std::max(s->max_obs, 1);
  const int mb = quad ? s->max_obs : (c->model == UCN_MODEL_MARS14 ? 6 : 3);
  const long long Xn = (long long)(s->Nmax + 1), Un = s->Nmax;
  s->state_per_slot = 6 * Xn * NX + 3 * Un * NU + 2 * Xn * mb * 3;
  const int tsize = c->precision == UCN_PREC_FP64 ? 8 : 4;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const long long static_sh = (long long)sizeof(InstShared) + 64;
  s->tpn = default_tpn(c->model, s->Nmax + 1, c->precision);
  s->L = make_layout(c->model, s->Nmax + 1, s->max_obs, tsize, c->model == UCN_MODEL_MARS7, s->tpn);
  s->smem = s->L.bytes + static_sh <= optin;
  if (!s->smem) {
    if (!tpn_allowed(s->tpn, c->model, s->Nmax + 1, c->precision, false)) s->tpn = 1;
    s->L = make_layout(c->model, s->Nmax + 1, s->max_obs, tsize, false, s->tpn);
  }
  s->smem_bytes = s->smem ? s->L.bytes : 0;
  s->threads = (s->Nmax + 1 + 31) / 32 * 32;
  s->R = c->kept > 0 ? c->kept : 2 * S;
  bool ok = true;
  ok = ok && halloc(s, &s->hN, S) && halloc(s, &s->hnobs, S) && halloc(s, &s->hdt, S) && halloc(s, &s->hprm, (size_t)S * 8);
  ok = ok && halloc(s, &s->hQd, (size_t)S * NX) && halloc(s, &s->hxr, (size_t)S * NX) && halloc(s, &s->hRd, (size_t)S * NU);
  ok = ok && halloc(s, &s->hur, (size_t)S * NU) && halloc(s, &s->hQNd, (size_t)S * NX) && halloc(s, &s->hqN, (size_t)S * NX);
  ok = ok && halloc(s, &s->hxlo, (size_t)S * NX) && halloc(s, &s->hxhi, (size_t)S * NX) && halloc(s, &s->hulo, (size_t)S * NU);
  ok = ok && halloc(s, &s->huhi, (size_t)S * NU) && halloc(s, &s->hxi, (size_t)S * NX) && halloc(s, &s->hxt, (size_t)S * NX);
  ok = ok && halloc(s, &s->htm, (size_t)S * NX) && halloc(s, &s->hoc, (size_t)S * MO * 3) && halloc(s, &s->hor, (size_t)S * MO);
  ok = ok && halloc(s, &s->hsets, (size_t)S * UCN_SET_PARAMS) && halloc(s, &s->hxg, (size_t)S * Xn * NX) && halloc(s, &s->hug, (size_t)S * Un * NU);
  ok = ok && dalloc(s, &s->dN, S) && dalloc(s, &s->dnobs, S) && dalloc(s, &s->ddt, S) && dalloc(s, &s->dprm, (size_t)S * 8);
  ok = ok && dalloc(s, &s->dQd, (size_t)S * NX) && dalloc(s, &s->dxr, (size_t)S * NX) && dalloc(s, &s->dRd, (size_t)S * NU);
  ok = ok && dalloc(s, &s->dur, (size_t)S * NU) && dalloc(s, &s->dQNd, (size_t)S * NX) && dalloc(s, &s->dqN, (size_t)S * NX);
  ok = ok && dalloc(s, &s->dxlo, (size_t)S * NX) && dalloc(s, &s->dxhi, (size_t)S * NX) && dalloc(s, &s->dulo, (size_t)S * NU);
  ok = ok && dalloc(s, &s->duhi, (size_t)S * NU) && dalloc(s, &s->dxi, (size_t)S * NX) && dalloc(s, &s->dxt, (size_t)S * NX);
  ok = ok && dalloc(s, &s->dtm, (size_t)S * NX) && dalloc(s, &s->doc, (size_t)S * MO * 3) && dalloc(s, &s->dor, (size_t)S * MO);
  ok = ok && dalloc(s, &s->dsets, (size_t)S * UCN_SET_PARAMS);
  ok = ok && dalloc(s, &s->x0, (size_t)S * Xn * NX) && dalloc(s, &s->u0, (size_t)S * Un * NU);
  ok = ok && dalloc(s, &s->xo, (size_t)S * Xn * NX) && dalloc(s, &s->uo, (size_t)S * Un * NU);
  ok = ok && dalloc(s, &s->stats, (size_t)S) && dalloc(s, &s->status, (size_t)S);
  ok = ok && dalloc(s, &s->ring_x, (size_t)s->R * Xn * NX) && dalloc(s, &s->ring_u, (size_t)s->R * Un * NU);
  long long *dxoff = nullptr, *duoff = nullptr, *dsoff = nullptr;
  double *sabs = nullptr, *dfac = nullptr;
  ok = ok && dalloc(s, &dxoff, S) && dalloc(s, &duoff, S) && dalloc(s, &dsoff, S) && dalloc(s, &sabs, (size_t)S * s->state_per_slot);
  const std::vector<double> fac = rho_schedule(c->rho_final, c->rho_geo, c->scp_iters);
  ok = ok && dalloc(s, &dfac, fac.size());
  char* ws = nullptr;
  if (ok && !s->smem) ok = dalloc(s, &ws, (size_t)s->L.bytes * S);
  if (ok) {
    std::vector<long long> xo(S), uo(S), so(S);
    for (int i = 0; i < S; ++i) { xo[i] = i * Xn; uo[i] = i * Un; so[i] = i * s->state_per_slot; }
    cudaMemcpy(dxoff, xo.data(), sizeof(long long) * S, cudaMemcpyHostToDevice);
    cudaMemcpy(duoff, uo.data(), sizeof(long long) * S, cudaMemcpyHostToDevice);
    cudaMemcpy(dsoff, so.data(), sizeof(long long) * S, cudaMemcpyHostToDevice);
    cudaMemcpy(dfac, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice);
    for (int l = 0; l < s->lanes && ok; ++l) {
      cudaStream_t st; cudaEvent_t ev; int *od, *oh;
      ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
           dalloc(s, &od, S) && halloc(s, &oh, S);
      if (ok) { s->streams.push_back(st); s->done.push_back(ev); s->order_d.push_back(od); s->order_h.push_back(oh); s->lane_busy.push_back(0); }
    }
  }
  if (!ok) { ucn_serve_destroy(s); return sfail(UCN_ENOMEM, "server allocation failed"); }
  ProblemDev& P = s->P;
  std::memset(&P, 0, sizeof(P));
  P.model = c->model; P.nx = NX; P.nu = NU; P.batch = S; P.max_obs = s->max_obs;
  P.N = s->dN; P.xoff = dxoff; P.uoff = duoff; P.soff = dsoff; P.dt = s->ddt; P.params = s->dprm;
  P.Qd = s->dQd; P.xref = s->dxr; P.Rd = s->dRd; P.uref = s->dur; P.QNd = s->dQNd; P.qN = s->dqN;
  P.xlo = s->dxlo; P.xhi = s->dxhi; P.ulo = s->dulo; P.uhi = s->duhi; P.xinit = s->dxi; P.xtarget = s->dxt;
  P.tmask = s->dtm; P.nobs = s->dnobs; P.obs_c = s->doc; P.obs_r = s->dor; P.sets = s->dsets;
  P.rho_eq = c->rho_eq; P.rho_dyn = c->rho_dyn; P.rho_geo = c->rho_geo; P.rho_final = c->rho_final;
  P.scp_iters = c->scp_iters; P.admm_iters = c->admm_iters; P.stop = c->stop;
  P.tr_init = c->tr_init; P.tr_min = c->tr_min; P.tr_max = c->tr_max; P.w_d = c->w_d;
  P.defect_tol = c->defect_tol; P.step_tol = c->step_tol;
  P.timeout_ns = (unsigned long long)((c->timeout_s > 0 ? c->timeout_s : 60.0) * 1e9);
  P.state_abs = sabs; P.ws = ws; P.order = nullptr; P.rho_fac = dfac;
  s->slot_state.assign(S, SLOT_FREE); s->slot_lane.assign(S, -1); s->slot_warm_ring.assign(S, -1);
  s->slot_ticket.assign(S, 0); s->slot_bytes.assign(S, 0);
  s->ring_ticket.assign(s->R, 0); s->ring_N.assign(s->R, 0); s->ring_next = 0;
  s->next_ticket = 1; s->used = 0;
  s->budget = c->hbm_budget_bytes > 0 ? (long long)c->hbm_budget_bytes : (long long)1 << 62;
  *out = s;
  return UCN_OK;
}

ucn_status ucn_serve_submit(ucn_server* s, const ucn_request* r, unsigned long long* ticket) {
  set_error_message("");
  if (!s || !r || !ticket) return sfail(UCN_EINVAL, "null argument");
  const int NX = s->nx, NU = s->nu, N = r->horizon;
  if (N < 1 || N > s->Nmax) return sfail(UCN_EINVAL, "horizon %d outside [1, %d]", N, s->Nmax);
  if (!(r->dt > 0) || !r->model_params || !r->Q_diag || !r->x_ref || !r->R_diag || !r->u_ref || !r->QN_diag || !r->qN ||
      !r->x_lo || !r->x_hi || !r->u_lo || !r->u_hi || !r->x_init || !r->x_target || !r->term_mask)
    return sfail(UCN_EINVAL, "incomplete request");
  if (model_obstacles(s->cfg.model) && (r->n_obs < 0 || r->n_obs > s->max_obs || (r->n_obs > 0 && (!r->obs_c || !r->obs_r))))
    return sfail(UCN_EINVAL, "bad obstacle data");
  if (!model_obstacles(s->cfg.model) && !r->sets) return sfail(UCN_EINVAL, "Mars requests need sets");
  std::lock_guard<std::mutex> lk(s->mu);
  int ring = -1;
  if (!(r->x_guess && r->u_guess)) {
    for (int k = 0; k < s->R; ++k)
      if (s->ring_ticket[k] == r->warm_ticket && r->warm_ticket != 0 && s->ring_N[k] == N) ring = k;
    if (ring < 0) return sfail(UCN_EINVAL, "no guess and no kept trajectory of horizon %d for ticket %llu", N, r->warm_ticket);
  }
  const long long fp = footprint(s, N);
  int slot = -1;
  for (int k = 0; k < s->S; ++k)
    if (s->slot_state[k] == SLOT_FREE) { slot = k; break; }
  if (slot < 0) return sfail(UCN_EBUSY, "no free slot");
  if (s->used + fp > s->budget) return sfail(UCN_EBUSY, "HBM budget: %lld of %lld bytes in use, request needs %lld", s->used, s->budget, fp);
  const int k = slot, MO = std::max(s->max_obs, 1);
  s->hN[k] = N; s->hdt[k] = r->dt;
  std::memcpy(&s->hprm[k * 8], r->model_params, 8 * sizeof(double));
  std::memcpy(&s->hQd[k * NX], r->Q_diag, NX * 8); std::memcpy(&s->hxr[k * NX], r->x_ref, NX * 8);
  std::memcpy(&s->hRd[k * NU], r->R_diag, NU * 8); std::memcpy(&s->hur[k * NU], r->u_ref, NU * 8);
  std::memcpy(&s->hQNd[k * NX], r->QN_diag, NX * 8); std::memcpy(&s->hqN[k * NX], r->qN, NX * 8);
  std::memcpy(&s->hxlo[k * NX], r->x_lo, NX * 8); std::memcpy(&s->hxhi[k * NX], r->x_hi, NX * 8);
  std::memcpy(&s->hulo[k * NU], r->u_lo, NU * 8); std::memcpy(&s->huhi[k * NU], r->u_hi, NU * 8);
  std::memcpy(&s->hxi[k * NX], r->x_init, NX * 8); std::memcpy(&s->hxt[k * NX], r->x_target, NX * 8);
  std::memcpy(&s->htm[k * NX], r->term_mask, NX);
  s->hnobs[k] = model_obstacles(s->cfg.model) ? r->n_obs : 0;
  if (s->hnobs[k] > 0) {
    std::memcpy(&s->hoc[(size_t)k * MO * 3], r->obs_c, (size_t)r->n_obs * 3 * 8);
    std::memcpy(&s->hor[(size_t)k * MO], r->obs_r, (size_t)r->n_obs * 8);
  }
  if (r->sets) std::memcpy(&s->hsets[k * UCN_SET_PARAMS], r->sets, UCN_SET_PARAMS * 8);
  else std::memset(&s->hsets[k * UCN_SET_PARAMS], 0, UCN_SET_PARAMS * 8);
  const long long Xn = s->Nmax + 1, Un = s->Nmax;
  if (ring < 0) {
    std::memcpy(&s->hxg[k * Xn * NX], r->x_guess, (size_t)(N + 1) * NX * 8);
    std::memcpy(&s->hug[k * Un * NU], r->u_guess, (size_t)N * NU * 8);
  }
  s->slot_warm_ring[k] = ring;
  s->slot_state[k] = SLOT_ADMITTED;
  s->slot_bytes[k] = fp;
  s->used += fp;
  s->slot_ticket[k] = s->next_ticket++;
  s->ticket_slot[s->slot_ticket[k]] = k;
  *ticket = s->slot_ticket[k];
  return UCN_OK;
}

ucn_status ucn_serve_pump(ucn_server* s, int* launched) {
  set_error_message("");
  if (!s) return sfail(UCN_EINVAL, "null server");
  if (launched) *launched = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<int> ready;
  for (int k = 0; k < s->S; ++k)
    if (s->slot_state[k] == SLOT_ADMITTED) ready.push_back(k);
  if (ready.empty()) return UCN_OK;
  int lane = -1;
  for (int l = 0; l < s->lanes; ++l) {
    if (s->lane_busy[l] && cudaEventQuery(s->done[l]) == cudaSuccess) s->lane_busy[l] = 0;
    if (!s->lane_busy[l] && lane < 0) lane = l;
  }
  if (lane < 0) return sfail(UCN_EBUSY, "every lane is running a launch");
  cudaStream_t st = s->streams[lane];
  const int S = s->S, NX = s->nx, NU = s->nu, MO = std::max(s->max_obs, 1);
  const long long Xn = s->Nmax + 1, Un = s->Nmax;
  // whole per-slot arrays from the pinned mirrors (running slots get their own, unchanged, bytes)
#define H2D(d, h, n) cudaMemcpyAsync(d, h, (size_t)(n) * sizeof(*(h)), cudaMemcpyHostToDevice, st)
  H2D(s->dN, s->hN, S); H2D(s->dnobs, s->hnobs, S); H2D(s->ddt, s->hdt, S); H2D(s->dprm, s->hprm, S * 8);
  H2D(s->dQd, s->hQd, S * NX); H2D(s->dxr, s->hxr, S * NX); H2D(s->dRd, s->hRd, S * NU); H2D(s->dur, s->hur, S * NU);
  H2D(s->dQNd, s->hQNd, S * NX); H2D(s->dqN, s->hqN, S * NX); H2D(s->dxlo, s->hxlo, S * NX); H2D(s->dxhi, s->hxhi, S * NX);
  H2D(s->dulo, s->hulo, S * NU); H2D(s->duhi, s->huhi, S * NU); H2D(s->dxi, s->hxi, S * NX); H2D(s->dxt, s->hxt, S * NX);
  H2D(s->dtm, s->htm, S * NX); H2D(s->doc, s->hoc, (size_t)S * MO * 3); H2D(s->dor, s->hor, (size_t)S * MO); H2D(s->dsets, s->hsets, S * UCN_SET_PARAMS);
  for (size_t j = 0; j < ready.size(); ++j) {
    const int k = ready[j], N = s->hN[k], ring = s->slot_warm_ring[k];
    if (ring >= 0) {
      cudaMemcpyAsync(&s->x0[k * Xn * NX], &s->ring_x[ring * Xn * NX], (size_t)(N + 1) * NX * 8, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(&s->u0[k * Un * NU], &s->ring_u[ring * Un * NU], (size_t)N * NU * 8, cudaMemcpyDeviceToDevice, st);
    } else {
      H2D(&s->x0[k * Xn * NX], &s->hxg[k * Xn * NX], (N + 1) * NX);
      H2D(&s->u0[k * Un * NU], &s->hug[k * Un * NU], N * NU);
    }
    s->order_h[lane][j] = k;
  }
  H2D(s->order_d[lane], s->order_h[lane], ready.size());
#undef H2D
  ProblemDev P = s->P;
  P.order = s->order_d[lane];
  LaunchCfg c;
  c.P = &P; c.L = &s->L; c.smem = s->smem; c.smem_bytes = s->smem_bytes;
  c.threads = s->threads; c.blocks = (int)ready.size(); c.stream = st; c.group = 1;
  c.nodes = s->cfg.max_horizon + 1; c.tpn = s->tpn;
  auto fn = launchers_for(s->cfg.model, s->cfg.precision).scp;
  cudaError_t e = fn(c, s->x0, s->u0, s->xo, s->uo, s->stats, s->status);
  if (e == cudaSuccess) e = cudaEventRecord(s->done[lane], st);
  if (e != cudaSuccess) return sfail(UCN_ECUDA, "serve launch: %s", cudaGetErrorString(e));
  s->lane_busy[lane] = 1;
  for (int k : ready) { s->slot_state[k] = SLOT_RUNNING; s->slot_lane[k] = lane; }
  if (launched) *launched = (int)ready.size();
  return UCN_OK;
}

ucn_status ucn_serve_poll(ucn_server* s, unsigned long long ticket, ucn_result* res) {
  set_error_message("");
  if (!s || !res) return sfail(UCN_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->ticket_slot.find(ticket);
  if (it == s->ticket_slot.end()) return sfail(UCN_EINVAL, "unknown ticket %llu", ticket);
  const int k = it->second;
  if (s->slot_state[k] != SLOT_RUNNING) return UCN_EBUSY;                 // admitted, not launched yet
  const int lane = s->slot_lane[k];
  const cudaError_t q = cudaEventQuery(s->done[lane]);
  if (q == cudaErrorNotReady) return UCN_EBUSY;
  if (q != cudaSuccess) return sfail(UCN_ECUDA, "serve launch failed: %s", cudaGetErrorString(q));
  const int NX = s->nx, NU = s->nu, N = s->hN[k];
  const long long Xn = s->Nmax + 1, Un = s->Nmax;
  cudaError_t e = cudaMemcpy(&res->stats, &s->stats[k], sizeof(ucn_scp_stats), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && res->x) e = cudaMemcpy(res->x, &s->xo[k * Xn * NX], (size_t)(N + 1) * NX * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && res->u) e = cudaMemcpy(res->u, &s->uo[k * Un * NU], (size_t)N * NU * 8, cudaMemcpyDeviceToHost);
  // keep the trajectory on the device for warm starts of later requests
  const int ring = s->ring_next;
  s->ring_next = (s->ring_next + 1) % s->R;
  if (e == cudaSuccess) e = cudaMemcpy(&s->ring_x[ring * Xn * NX], &s->xo[k * Xn * NX], (size_t)(N + 1) * NX * 8, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(&s->ring_u[ring * Un * NU], &s->uo[k * Un * NU], (size_t)N * NU * 8, cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) return sfail(UCN_ECUDA, "result copy: %s", cudaGetErrorString(e));
  s->ring_ticket[ring] = ticket;
  s->ring_N[ring] = N;
  res->ticket = ticket;
  res->horizon = N;
  s->slot_state[k] = SLOT_FREE;
  s->used -= s->slot_bytes[k];
  s->ticket_slot.erase(it);
  return UCN_OK;
}

int ucn_serve_free_slots(ucn_server* s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  for (int v : s->slot_state) n += (v == SLOT_FREE);
  return n;
}

}  // extern "C"
