// Serving: continuous batching of SCP solves over a preallocated slot pool.
//
// All device memory is allocated once by ucn_serve_create, for `max_slots`
// instances of up to `max_horizon` nodes (problem data, guesses, outputs,
// exported ADMM state, workspace) plus a ring of kept results -- trajectory
// and final ADMM state -- for warm starts.  Requests are admitted into free
// slots while their HBM footprint fits the budget; every pump launches the
// fused SCP kernel over the slots admitted since the last pump, on the next
// free lane (a CUDA stream), while earlier launches keep running on the other
// lanes.  Each instance's solve is independent of the others in its launch
// (one CTA per instance, same CTA size and layout for every slot), so a result
// does not depend on what it was batched with.
//
// Data movement of a launch, all on its lane's stream: the admitted requests'
// records (problem data and guesses) go up in ONE copy from a pinned staging
// buffer and a scatter kernel writes them into the slot arrays (a warm request
// instead takes its guess and ADMM state from the ring entry of the request it
// names).  Each CTA of the solve writes its own result (stats, x, u) into its
// slot's record in mapped host memory the moment its instance is done and then
// raises the slot's flag (deliver_result), so a request's result is available
// when ITS solve ends, not when the launch's slowest one does; after the solve
// a keep kernel copies the launch's trajectories and final ADMM states into the
// ring.  ucn_serve_poll and ucn_serve_poll_any read host memory only.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "ucn_internal.h"
#include "ucn_serve.cuh"

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

// A slot is FREE, ADMITTED (waiting for a pump), RUNNING (launched), or
// DRAINING: its result was taken but its launch's keep kernel may still read
// its device arrays, so it is not reused before that launch ends.
enum { SLOT_FREE = 0, SLOT_ADMITTED = 1, SLOT_RUNNING = 2, SLOT_DRAINING = 3 };
// slot_lane / ring_lane of a request published to the device-resident loop
constexpr int LOOP_LANE = -2;

// Requests per launch (bounds the pinned staging of a lane).
constexpr int LAUNCH_CAP = 128;

// One CTA per launched request j: its record rec[j] into the slot arrays (or
// the guess and ADMM state from a ring entry for a warm start), and the CTA ->
// slot order of the launch.
__global__ void serve_scatter_kernel(ServeDev D, const double* rec, int* order) {
  const int k = serve_scatter_one<false>(D, rec + (long long)blockIdx.x * D.REC);
  if (threadIdx.x == 0) order[blockIdx.x] = k;
}

// One CTA per launched request j that keeps its result: its trajectory and
// final ADMM state into the ring entry the launch assigned it (warm starts).
__global__ void serve_keep_kernel(ServeDev D, const double* rec) {
  serve_keep_one<false>(D, rec + (long long)blockIdx.x * D.REC);
}

}  // namespace

struct ucn_server {
  ucn_serve_config cfg;
  int nx, nu, S, Nmax, max_obs, lanes, MO;
  long long state_per_slot, budget, used;
  int nalloc = 0, fault_at = 0;   // allocations made by create; UCN_FAULT_ALLOC
  ProblemDev P;
  ServeDev D;
  RecLayout rl;
  Layout L;
  bool smem;
  long long smem_bytes;
  int threads;
  int tpn;               // threads per node of the fused solve
  int* status_d;         // per-slot status of the fused solve
  std::vector<void*> dev_allocs, host_allocs;
  std::vector<double> hrec;          // admitted requests' records, [S][REC] (host)
  // slots
  std::vector<int> slot_state, slot_lane, slot_pos, slot_ring_read, slot_ring_write;
  std::vector<unsigned long long> slot_ticket;
  std::vector<long long> slot_bytes;
  std::map<unsigned long long, int> ticket_slot;
  unsigned long long next_ticket;
  // results: per-slot records and flags in mapped host memory (host and device views)
  double *res_h, *res_dv;
  unsigned long long *flag_h, *flag_dv;
  // lanes: stream, completion event, staging (pinned host, device), the ring
  // entries its running launch fills, a launch failure
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  std::vector<double*> stage_h, stage_d;
  std::vector<int*> order_d;
  std::vector<int> lane_busy;
  std::vector<cudaError_t> lane_error;
  std::vector<std::vector<int>> lane_rings;
  // ring of kept results: ticket, horizon, kept (its launch has finished),
  // being written (by lane ring_lane), admitted requests reading it
  int R, ring_next;
  std::vector<unsigned long long> ring_ticket;
  std::vector<int> ring_N, ring_done, ring_writing, ring_lane, ring_readers;
  // the device-resident request loop: per-slot request records, the queue of
  // published slots and its head, the stop flag (mapped host memory; host and
  // device views), the claim counter (device memory), its stream and the event
  // recorded after its launch
  double *lrec_h = nullptr, *lrec_dv = nullptr;
  long long *lq_h = nullptr, *lq_dv = nullptr;
  unsigned long long *lhead_h = nullptr, *lhead_dv = nullptr;
  unsigned *lstop_h = nullptr, *lstop_dv = nullptr;
  unsigned long long* lnext_d = nullptr;
  cudaStream_t loop_stream = nullptr;
  cudaEvent_t loop_done = nullptr;
  bool loop_on = false;         // submit publishes to the loop (ucn_serve_loop_start .. _stop)
  bool loop_live = false;       // a loop launch has been made and not seen to end
  int loop_ctas = 0;            // CTAs asked for (0: every CTA that can be resident)
  unsigned long long loop_idle_ns = 0;
  unsigned long long published = 0;
  cudaError_t loop_error = cudaSuccess;
  int loop_launches = 0, loop_ctas_launched = 0;
  std::mutex mu;
};

namespace {

template <class V>
bool dalloc(ucn_server* s, V** out, size_t n) {
  if (++s->nalloc == s->fault_at) return false;
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n * sizeof(V), 16)) != cudaSuccess) { cudaGetLastError(); return false; }
  cudaMemset(p, 0, std::max<size_t>(n * sizeof(V), 16));
  s->dev_allocs.push_back(p);
  *out = (V*)p;
  return true;
}

template <class V>
bool halloc(ucn_server* s, V** out, size_t n) {
  if (++s->nalloc == s->fault_at) return false;
  void* p = nullptr;
  if (cudaMallocHost(&p, std::max<size_t>(n * sizeof(V), 16)) != cudaSuccess) { cudaGetLastError(); return false; }
  std::memset(p, 0, std::max<size_t>(n * sizeof(V), 16));
  s->host_allocs.push_back(p);
  *out = (V*)p;
  return true;
}

// Pinned host memory the device writes directly (mapped): host and device views.
template <class V>
bool mapped(ucn_server* s, V** host, V** dev, size_t n) {
  if (++s->nalloc == s->fault_at) return false;
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(n * sizeof(V), 16);
  if (cudaHostAlloc(&p, bytes, cudaHostAllocMapped) != cudaSuccess) { cudaGetLastError(); return false; }
  std::memset(p, 0, bytes);
  s->host_allocs.push_back(p);
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) { cudaGetLastError(); return false; }
  *host = (V*)p;
  *dev = (V*)d;
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

void release_slot(ucn_server* s, int k) {
  s->slot_state[k] = SLOT_FREE;
  s->used -= s->slot_bytes[k];
  s->slot_bytes[k] = 0;
}

// A lane whose launch has finished: the ring entries it filled become kept and
// its drained slots free.
void retire_lane(ucn_server* s, int l) {
  for (int r : s->lane_rings[l]) { s->ring_writing[r] = 0; s->ring_done[r] = 1; }
  s->lane_rings[l].clear();
  s->lane_busy[l] = 0;
  for (int k = 0; k < s->S; ++k)
    if (s->slot_state[k] == SLOT_DRAINING && s->slot_lane[k] == l) release_slot(s, k);
}


// Whether lane l's launch has ended (finished, or failed: lane_error).
bool lane_ended(ucn_server* s, int l) {
  if (!s->lane_busy[l]) return true;
  const cudaError_t q = cudaEventQuery(s->done[l]);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) s->lane_error[l] = q;
  retire_lane(s, l);
  return true;
}

// Retires every lane whose launch has ended.
void retire_ended(ucn_server* s) {
  for (int l = 0; l < s->lanes; ++l) lane_ended(s, l);
}

// A ring entry that no launch is writing and no admitted request reads, the
// oldest first (round robin); -1 when every entry is held.
int take_ring_entry(ucn_server* s) {
  for (int t = 0; t < s->R; ++t) {
    const int r = (s->ring_next + t) % s->R;
    if (!s->ring_writing[r] && s->ring_readers[r] == 0) {
      s->ring_next = (r + 1) % s->R;
      return r;
    }
  }
  return -1;
}

bool delivered(const ucn_server* s, int k);

// Publishes admitted slot k to the device-resident loop: the ring entry that
// keeps its result, its record into mapped memory, its queue entry, then the
// head (a release store: the GPU's acquire load of the head sees the rest).
void publish(ucn_server* s, int k) {
  const RecLayout& L = s->rl;
  double* rec = &s->hrec[(size_t)k * L.END];
  const int rw = take_ring_entry(s);
  rec[L.RINGW] = rw;
  s->slot_ring_write[k] = rw;
  if (rw >= 0) {
    s->ring_writing[rw] = 1; s->ring_done[rw] = 0; s->ring_lane[rw] = LOOP_LANE;
    s->ring_ticket[rw] = s->slot_ticket[k]; s->ring_N[rw] = (int)rec[L.N];
  }
  std::memcpy(s->lrec_h + (size_t)k * L.END, rec, (size_t)L.END * sizeof(double));
  s->lq_h[s->published % (unsigned long long)s->S] = k;
  ++s->published;
  __atomic_store_n(s->lhead_h, s->published, __ATOMIC_RELEASE);
  s->slot_state[k] = SLOT_RUNNING; s->slot_lane[k] = LOOP_LANE; s->slot_pos[k] = -1;
}

// Whether the loop launch has ended (recording a failure); false while it runs.
bool loop_ended(ucn_server* s) {
  if (!s->loop_live) return true;
  const cudaError_t q = cudaEventQuery(s->loop_done);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) s->loop_error = q;
  s->loop_live = false;
  return true;
}

// One launch of the loop kernel on the loop's stream (query: only the number
// of its CTAs that can be resident at once, into *cap).
cudaError_t loop_launch(ucn_server* s, bool query = false, int* cap = nullptr) {
  auto fn = loop_launcher_for(s->cfg.model, s->cfg.precision);
  if (!fn) return cudaErrorNotSupported;
  LoopDev Q;
  Q.rec = s->lrec_dv; Q.queue = s->lq_dv; Q.head = s->lhead_dv; Q.stop = s->lstop_dv; Q.next = s->lnext_d;
  Q.idle_ns = s->loop_idle_ns; Q.S = s->S;
  LoopCfg c;
  c.Q = &Q; c.D = &s->D; c.P = &s->P; c.L = &s->L; c.status = s->status_d;
  c.smem = s->smem; c.smem_bytes = s->smem_bytes;
  c.threads = s->tpn == 4 ? (4 * (s->Nmax + 1) + 31) / 32 * 32 : s->threads;
  c.tpn = s->tpn; c.ctas = s->loop_ctas; c.stream = s->loop_stream;
  int n = 0;
  c.launched_ctas = &n;
  c.query = query;
  cudaError_t e = fn(c);
  if (query) {
    if (cap) *cap = e == cudaSuccess ? n : 0;
    return e;
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->loop_done, s->loop_stream);
  if (e != cudaSuccess) { s->loop_error = e; return e; }
  s->loop_live = true;
  ++s->loop_launches;
  s->loop_ctas_launched = n;
  return cudaSuccess;
}

// A new loop launch when the last one has ended (its CTAs found no request for
// the idle time) while published requests wait; the loop's failure, if any.
cudaError_t loop_kick(ucn_server* s) {
  if (!s->loop_on || s->loop_error != cudaSuccess || !loop_ended(s) || s->loop_error != cudaSuccess)
    return s->loop_error;
  bool pending = false;
  for (int k = 0; k < s->S && !pending; ++k)
    pending = s->slot_state[k] == SLOT_RUNNING && s->slot_lane[k] == LOOP_LANE && !delivered(s, k);
  return pending ? loop_launch(s) : cudaSuccess;
}

// Whether ring entry r holds a complete result that a request published to the
// loop may read (the loop orders nothing by streams): its writer's launch has
// ended, or its writer is a loop request whose result has been delivered (the
// loop writes the ring entry before it delivers).
bool ring_complete(ucn_server* s, int r) {
  if (s->ring_done[r]) return true;
  if (!s->ring_writing[r]) return false;
  if (s->ring_lane[r] == LOOP_LANE) {
    auto it = s->ticket_slot.find(s->ring_ticket[r]);
    return it != s->ticket_slot.end() && delivered(s, it->second);
  }
  lane_ended(s, s->ring_lane[r]);   // retires the lane: its entries become kept
  return s->ring_done[r] != 0;
}

}  // namespace

extern "C" {

void ucn_serve_destroy(ucn_server* s) {
  if (!s) return;
  if (s->lstop_h) __atomic_store_n(s->lstop_h, 1u, __ATOMIC_RELEASE);   // a running loop ends
  cudaDeviceSynchronize();
  if (s->loop_stream) cudaStreamDestroy(s->loop_stream);
  if (s->loop_done) cudaEventDestroy(s->loop_done);
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
  s->fault_at = fault_alloc_at();
  const bool quad = model_obstacles(c->model);
  s->nx = model_nx(c->model); s->nu = model_nu(c->model);
  s->S = c->max_slots; s->Nmax = c->max_horizon; s->max_obs = quad ? c->max_obs : 0; s->lanes = c->lanes;
  const int S = s->S, NX = s->nx, NU = s->nu, MO = std::max(s->max_obs, 1);
  s->MO = MO;
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
  s->rl = rec_layout(NX, NU, MO, (int)Xn, (int)Un);
  const int REC = s->rl.END, RES = (int)((16 + Xn * NX + Un * NU + 1) / 2 * 2);
  const int cap = std::min(S, LAUNCH_CAP);
  ServeDev& D = s->D;
  std::memset(&D, 0, sizeof(D));
  D.NX = NX; D.NU = NU; D.MO = MO; D.Xn = (int)Xn; D.Un = (int)Un; D.REC = REC; D.RES = RES;
  D.state_per_slot = s->state_per_slot; D.rl = s->rl;
  bool ok = true;
  ok = ok && dalloc(s, &D.N, S) && dalloc(s, &D.nobs, S) && dalloc(s, &D.dt, S) && dalloc(s, &D.prm, (size_t)S * 8);
  ok = ok && dalloc(s, &D.Qd, (size_t)S * NX) && dalloc(s, &D.xr, (size_t)S * NX) && dalloc(s, &D.Rd, (size_t)S * NU);
  ok = ok && dalloc(s, &D.ur, (size_t)S * NU) && dalloc(s, &D.QNd, (size_t)S * NX) && dalloc(s, &D.qN, (size_t)S * NX);
  ok = ok && dalloc(s, &D.xlo, (size_t)S * NX) && dalloc(s, &D.xhi, (size_t)S * NX) && dalloc(s, &D.ulo, (size_t)S * NU);
  ok = ok && dalloc(s, &D.uhi, (size_t)S * NU) && dalloc(s, &D.xi, (size_t)S * NX) && dalloc(s, &D.xt, (size_t)S * NX);
  ok = ok && dalloc(s, &D.tm, (size_t)S * NX) && dalloc(s, &D.oc, (size_t)S * MO * 3) && dalloc(s, &D.orr, (size_t)S * MO);
  ok = ok && dalloc(s, &D.sets, (size_t)S * UCN_SET_PARAMS) && dalloc(s, &D.warm, (size_t)S) && dalloc(s, &D.tag, (size_t)S);
  ok = ok && dalloc(s, &D.x0, (size_t)S * Xn * NX) && dalloc(s, &D.u0, (size_t)S * Un * NU);
  ok = ok && dalloc(s, &D.xo, (size_t)S * Xn * NX) && dalloc(s, &D.uo, (size_t)S * Un * NU);
  ok = ok && dalloc(s, &D.stats, (size_t)S);
  ok = ok && dalloc(s, &D.state, (size_t)S * s->state_per_slot);
  ok = ok && dalloc(s, &D.ring_x, (size_t)s->R * Xn * NX) && dalloc(s, &D.ring_u, (size_t)s->R * Un * NU);
  ok = ok && dalloc(s, &D.ring_state, (size_t)s->R * s->state_per_slot);
  ok = ok && dalloc(s, &s->status_d, (size_t)S);
  // result records and flags in mapped host memory, written by the solve's CTAs
  ok = ok && mapped(s, &s->res_h, &s->res_dv, (size_t)S * RES) && mapped(s, &s->flag_h, &s->flag_dv, (size_t)S);
  // the request loop's records, queue, head and stop flag, claim counter
  ok = ok && mapped(s, &s->lrec_h, &s->lrec_dv, (size_t)S * REC) && mapped(s, &s->lq_h, &s->lq_dv, (size_t)S);
  ok = ok && mapped(s, &s->lhead_h, &s->lhead_dv, 1) && mapped(s, &s->lstop_h, &s->lstop_dv, 1);
  ok = ok && dalloc(s, &s->lnext_d, 1);
  if (ok) {
    ok = cudaStreamCreateWithFlags(&s->loop_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) s->loop_stream = nullptr;
  }
  if (ok) {
    ok = cudaEventCreateWithFlags(&s->loop_done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) s->loop_done = nullptr;
  }
  long long *dxoff = nullptr, *duoff = nullptr, *dsoff = nullptr;
  double* dfac = nullptr;
  ok = ok && dalloc(s, &dxoff, S) && dalloc(s, &duoff, S) && dalloc(s, &dsoff, S);
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
      // each resource is owned by the server as soon as it exists, so a failure
      // part way leaves nothing for destroy to miss
      cudaStream_t st; cudaEvent_t ev; int* od; double *sh, *sd;
      ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) s->streams.push_back(st);
      ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
      if (ok) s->done.push_back(ev);
      ok = ok && dalloc(s, &od, cap) && halloc(s, &sh, (size_t)cap * REC) && dalloc(s, &sd, (size_t)cap * REC);
      if (ok) {
        s->order_d.push_back(od); s->stage_h.push_back(sh); s->stage_d.push_back(sd);
        s->lane_busy.push_back(0); s->lane_error.push_back(cudaSuccess); s->lane_rings.emplace_back();
      }
    }
  }
  if (!ok) {
    const int fa = s->fault_at;
    const bool injected = fa > 0 && s->nalloc >= fa;
    ucn_serve_destroy(s);
    return injected ? sfail(UCN_ENOMEM, "injected allocation failure (UCN_FAULT_ALLOC=%d)", fa)
                    : sfail(UCN_ENOMEM, "server allocation failed");
  }
  s->hrec.assign((size_t)S * REC, 0.0);
  ProblemDev& P = s->P;
  std::memset(&P, 0, sizeof(P));
  P.model = c->model; P.nx = NX; P.nu = NU; P.batch = S; P.max_obs = s->max_obs;
  P.N = D.N; P.xoff = dxoff; P.uoff = duoff; P.soff = dsoff; P.dt = D.dt; P.params = D.prm;
  P.Qd = D.Qd; P.xref = D.xr; P.Rd = D.Rd; P.uref = D.ur; P.QNd = D.QNd; P.qN = D.qN;
  P.xlo = D.xlo; P.xhi = D.xhi; P.ulo = D.ulo; P.uhi = D.uhi; P.xinit = D.xi; P.xtarget = D.xt;
  P.tmask = D.tm; P.nobs = D.nobs; P.obs_c = D.oc; P.obs_r = D.orr; P.sets = D.sets;
  P.rho_eq = c->rho_eq; P.rho_dyn = c->rho_dyn; P.rho_geo = c->rho_geo; P.rho_final = c->rho_final;
  P.scp_iters = c->scp_iters; P.admm_iters = c->admm_iters; P.stop = c->stop;
  P.tr_init = c->tr_init; P.tr_min = c->tr_min; P.tr_max = c->tr_max; P.w_d = c->w_d;
  P.defect_tol = c->defect_tol; P.step_tol = c->step_tol;
  P.timeout_ns = (unsigned long long)((c->timeout_s > 0 ? c->timeout_s : 60.0) * 1e9);
  P.state_abs = D.state; P.ws = ws; P.order = nullptr; P.rho_fac = dfac; P.warm = D.warm;
  P.res_host = s->res_dv; P.res_flag = s->flag_dv; P.res_tag = D.tag; P.res_stride = RES;
  s->slot_state.assign(S, SLOT_FREE); s->slot_lane.assign(S, -1); s->slot_pos.assign(S, -1);
  s->slot_ring_read.assign(S, -1); s->slot_ring_write.assign(S, -1);
  s->slot_ticket.assign(S, 0); s->slot_bytes.assign(S, 0);
  s->ring_ticket.assign(s->R, 0); s->ring_N.assign(s->R, 0); s->ring_done.assign(s->R, 0);
  s->ring_writing.assign(s->R, 0); s->ring_lane.assign(s->R, -1); s->ring_readers.assign(s->R, 0); s->ring_next = 0;
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
      if (r->warm_ticket != 0 && s->ring_ticket[k] == r->warm_ticket && (s->ring_done[k] || s->ring_writing[k]) &&
          s->ring_N[k] == N)
        ring = k;
    if (ring < 0) return sfail(UCN_EINVAL, "no guess and no kept result of horizon %d for ticket %llu", N, r->warm_ticket);
    if (s->loop_on && !ring_complete(s, ring))
      return sfail(UCN_EBUSY, "the kept result of ticket %llu is not complete yet", r->warm_ticket);
  }
  const long long fp = footprint(s, N);
  int slot = -1;
  for (int pass = 0; pass < 2 && slot < 0; ++pass) {
    if (pass == 1 || s->used + fp > s->budget) retire_ended(s);   // frees drained slots
    for (int k = 0; k < s->S; ++k)
      if (s->slot_state[k] == SLOT_FREE) { slot = k; break; }
  }
  if (slot < 0) return sfail(UCN_EBUSY, "no free slot");
  if (s->used + fp > s->budget) return sfail(UCN_EBUSY, "HBM budget: %lld of %lld bytes in use, request needs %lld", s->used, s->budget, fp);
  const int k = slot;
  const RecLayout& L = s->rl;
  double* rec = &s->hrec[(size_t)k * L.END];
  std::fill(rec, rec + L.END, 0.0);
  rec[L.K] = k; rec[L.RING] = ring; rec[L.RINGW] = -1; rec[L.N] = N; rec[L.DT] = r->dt;
  rec[L.TAG] = (double)s->next_ticket;
  rec[L.NOBS] = model_obstacles(s->cfg.model) ? r->n_obs : 0;
  std::memcpy(&rec[L.PRM], r->model_params, 8 * sizeof(double));
  std::memcpy(&rec[L.QD], r->Q_diag, NX * 8); std::memcpy(&rec[L.XR], r->x_ref, NX * 8);
  std::memcpy(&rec[L.RD], r->R_diag, NU * 8); std::memcpy(&rec[L.UR], r->u_ref, NU * 8);
  std::memcpy(&rec[L.QND], r->QN_diag, NX * 8); std::memcpy(&rec[L.QN], r->qN, NX * 8);
  std::memcpy(&rec[L.XLO], r->x_lo, NX * 8); std::memcpy(&rec[L.XHI], r->x_hi, NX * 8);
  std::memcpy(&rec[L.ULO], r->u_lo, NU * 8); std::memcpy(&rec[L.UHI], r->u_hi, NU * 8);
  std::memcpy(&rec[L.XI], r->x_init, NX * 8); std::memcpy(&rec[L.XT], r->x_target, NX * 8);
  for (int j = 0; j < NX; ++j) rec[L.TM + j] = r->term_mask[j];
  if (rec[L.NOBS] > 0) {
    std::memcpy(&rec[L.OC], r->obs_c, (size_t)r->n_obs * 3 * 8);
    std::memcpy(&rec[L.OR], r->obs_r, (size_t)r->n_obs * 8);
  }
  if (r->sets) std::memcpy(&rec[L.SETS], r->sets, UCN_SET_PARAMS * 8);
  if (ring < 0) {
    std::memcpy(&rec[L.XG], r->x_guess, (size_t)(N + 1) * NX * 8);
    std::memcpy(&rec[L.UG], r->u_guess, (size_t)N * NU * 8);
  } else {
    s->ring_readers[ring]++;   // held until this request's result is collected
  }
  s->slot_ring_read[k] = ring;
  s->slot_state[k] = SLOT_ADMITTED;
  s->slot_bytes[k] = fp;
  s->used += fp;
  s->slot_ticket[k] = s->next_ticket++;
  s->ticket_slot[s->slot_ticket[k]] = k;
  *ticket = s->slot_ticket[k];
  if (s->loop_on) {
    publish(s, k);
    const cudaError_t e = loop_kick(s);
    if (e != cudaSuccess) return sfail(UCN_ECUDA, "request loop: %s", cudaGetErrorString(e));
  }
  return UCN_OK;
}

ucn_status ucn_serve_pump(ucn_server* s, int* launched) {
  set_error_message("");
  if (!s) return sfail(UCN_EINVAL, "null server");
  if (launched) *launched = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->loop_on) {   // requests go to the loop at submit; relaunch it if it ended idle
    const cudaError_t e = loop_kick(s);
    return e == cudaSuccess ? UCN_OK : sfail(UCN_ECUDA, "request loop: %s", cudaGetErrorString(e));
  }
  std::vector<int> ready;
  const int cap = std::min(s->S, LAUNCH_CAP);
  for (int k = 0; k < s->S && (int)ready.size() < cap; ++k)
    if (s->slot_state[k] == SLOT_ADMITTED) ready.push_back(k);
  if (ready.empty()) return UCN_OK;
  // a free lane: its last launch has ended
  int lane = -1;
  for (int l = 0; l < s->lanes; ++l)
    if (lane_ended(s, l) && lane < 0) lane = l;
  if (lane < 0) return sfail(UCN_EBUSY, "every lane is running a launch");
  s->lane_error[lane] = cudaSuccess;
  cudaStream_t st = s->streams[lane];
  const RecLayout& L = s->rl;
  const int n = (int)ready.size();
  double* stage = s->stage_h[lane];
  for (int j = 0; j < n; ++j) {
    const int k = ready[j];
    double* rec = &s->hrec[(size_t)k * L.END];
    const int rw = take_ring_entry(s);   // where this request's result is kept for warm starts
    rec[L.RINGW] = rw;
    s->slot_ring_write[k] = rw;
    if (rw >= 0) {
      s->ring_writing[rw] = 1; s->ring_done[rw] = 0; s->ring_lane[rw] = lane;
      s->ring_ticket[rw] = s->slot_ticket[k]; s->ring_N[rw] = (int)rec[L.N];
      s->lane_rings[lane].push_back(rw);
    }
    std::memcpy(stage + (size_t)j * L.END, rec, (size_t)L.END * sizeof(double));
  }
  cudaError_t e = cudaSuccess;
  // a warm request whose ring entry another lane is still filling reads it after that lane's launch
  for (int k : ready) {
    const int rr = s->slot_ring_read[k];
    if (rr >= 0 && s->ring_writing[rr] && s->ring_lane[rr] != lane && e == cudaSuccess)
      e = cudaStreamWaitEvent(st, s->done[s->ring_lane[rr]], 0);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->stage_d[lane], stage, (size_t)n * L.END * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    serve_scatter_kernel<<<n, 128, 0, st>>>(s->D, s->stage_d[lane], s->order_d[lane]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProblemDev P = s->P;
    P.order = s->order_d[lane];
    LaunchCfg c;
    c.P = &P; c.L = &s->L; c.smem = s->smem; c.smem_bytes = s->smem_bytes;
    c.threads = s->threads; c.blocks = n; c.stream = st; c.group = 1;
    c.nodes = s->cfg.max_horizon + 1; c.tpn = s->tpn;
    auto fn = launchers_for(s->cfg.model, s->cfg.precision).scp;
    e = fn(c, s->D.x0, s->D.u0, s->D.xo, s->D.uo, s->D.stats, s->status_d);
  }
  if (e == cudaSuccess) {
    serve_keep_kernel<<<n, 128, 0, st>>>(s->D, s->stage_d[lane]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->done[lane], st);
  if (e != cudaSuccess) {
    for (int k : ready)
      if (s->slot_ring_write[k] >= 0) { s->ring_writing[s->slot_ring_write[k]] = 0; s->slot_ring_write[k] = -1; }
    s->lane_rings[lane].clear();
    return sfail(UCN_ECUDA, "serve launch: %s", cudaGetErrorString(e));
  }
  s->lane_busy[lane] = 1;
  for (int j = 0; j < n; ++j) {
    const int k = ready[j];
    s->slot_state[k] = SLOT_RUNNING; s->slot_lane[k] = lane; s->slot_pos[k] = j;
  }
  if (launched) *launched = n;
  return UCN_OK;
}

}  // extern "C"

namespace {

// The finished request in slot k (its flag carries its ticket) into res; frees
// the slot.  Host memory only.
void take_result(ucn_server* s, int k, ucn_result* res) {
  const int NX = s->nx, NU = s->nu, N = (int)s->hrec[(size_t)k * s->rl.END + s->rl.N];
  const double* o = s->res_h + (size_t)k * s->D.RES;
  std::memcpy(&res->stats, o, sizeof(ucn_scp_stats));
  if (res->x) std::memcpy(res->x, o + 16, (size_t)(N + 1) * NX * sizeof(double));
  if (res->u) std::memcpy(res->u, o + 16 + (N + 1) * NX, (size_t)N * NU * sizeof(double));
  const int rr = s->slot_ring_read[k], rw = s->slot_ring_write[k];
  if (rr >= 0) s->ring_readers[rr]--;   // its launch read the entry before the solve began
  s->slot_ring_write[k] = s->slot_ring_read[k] = -1;
  res->ticket = s->slot_ticket[k];
  res->horizon = N;
  s->ticket_slot.erase(s->slot_ticket[k]);
  if (s->slot_lane[k] == LOOP_LANE) {
    // the loop's CTA kept the result and left the slot before it delivered
    if (rw >= 0) { s->ring_writing[rw] = 0; s->ring_done[rw] = 1; }
    release_slot(s, k);
  } else if (s->lane_busy[s->slot_lane[k]]) {
    s->slot_state[k] = SLOT_DRAINING;   // freed when its lane retires
  } else {
    release_slot(s, k);
  }
}

// Slot k's request has been delivered (its CTA raised the flag with its ticket).
bool delivered(const ucn_server* s, int k) {
  if (s->slot_state[k] != SLOT_RUNNING || *(volatile const unsigned long long*)(s->flag_h + k) != s->slot_ticket[k])
    return false;
  std::atomic_thread_fence(std::memory_order_acquire);   // the record was written before the flag
  return true;
}

}  // namespace

extern "C" {

ucn_status ucn_serve_poll(ucn_server* s, unsigned long long ticket, ucn_result* res) {
  set_error_message("");
  if (!s || !res) return sfail(UCN_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->ticket_slot.find(ticket);
  if (it == s->ticket_slot.end()) return sfail(UCN_EINVAL, "unknown ticket %llu", ticket);
  const int k = it->second;
  if (!delivered(s, k)) {
    if (s->slot_state[k] == SLOT_RUNNING) {
      const int l = s->slot_lane[k];
      if (l == LOOP_LANE) {
        const cudaError_t e = loop_kick(s);
        if (e != cudaSuccess && !delivered(s, k))
          return sfail(UCN_ECUDA, "request loop failed: %s", cudaGetErrorString(e));
      } else if (lane_ended(s, l) && !delivered(s, k) && s->lane_error[l] != cudaSuccess) {
        return sfail(UCN_ECUDA, "serve launch failed: %s", cudaGetErrorString(s->lane_error[l]));
      }
    }
    if (!delivered(s, k)) return UCN_EBUSY;   // admitted and not launched yet, or still solving
  }
  take_result(s, k, res);
  return UCN_OK;
}

ucn_status ucn_serve_poll_any(ucn_server* s, ucn_result* res) {
  set_error_message("");
  if (!s || !res) return sfail(UCN_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  for (int k = 0; k < s->S; ++k)
    if (delivered(s, k)) {
      take_result(s, k, res);
      return UCN_OK;
    }
  // nothing delivered: retire the lanes whose launches ended (their ring entries
  // become kept) and report a failed launch
  for (int l = 0; l < s->lanes; ++l)
    if (lane_ended(s, l) && s->lane_error[l] != cudaSuccess)
      return sfail(UCN_ECUDA, "serve launch failed: %s", cudaGetErrorString(s->lane_error[l]));
  const cudaError_t e = loop_kick(s);
  if (e != cudaSuccess) return sfail(UCN_ECUDA, "request loop failed: %s", cudaGetErrorString(e));
  return UCN_EBUSY;
}

ucn_status ucn_serve_loop_start(ucn_server* s, int ctas, double idle_s) {
  set_error_message("");
  if (!s) return sfail(UCN_EINVAL, "null server");
  if (!loop_launcher_for(s->cfg.model, s->cfg.precision)) return sfail(UCN_EINVAL, "no request loop for this model");
  if (ctas < 0 || !(idle_s > 0.0 && idle_s <= 60.0)) return sfail(UCN_EINVAL, "ctas must be >= 0 and idle_s in (0, 60]");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->loop_on) return sfail(UCN_EINVAL, "the request loop is already on");
  s->loop_ctas = ctas;
  s->loop_idle_ns = (unsigned long long)(idle_s * 1e9);
  s->loop_error = cudaSuccess;
  __atomic_store_n(s->lstop_h, 0u, __ATOMIC_RELEASE);
  s->loop_on = true;
  // requests admitted and not pumped go to the loop, oldest first
  std::vector<std::pair<unsigned long long, int>> adm;
  for (int k = 0; k < s->S; ++k)
    if (s->slot_state[k] == SLOT_ADMITTED) adm.emplace_back(s->slot_ticket[k], k);
  std::sort(adm.begin(), adm.end());
  for (auto& a : adm) publish(s, a.second);
  const cudaError_t e = loop_launch(s);
  if (e != cudaSuccess) return sfail(UCN_ECUDA, "request loop launch: %s", cudaGetErrorString(e));
  return UCN_OK;
}

ucn_status ucn_serve_loop_stop(ucn_server* s) {
  set_error_message("");
  if (!s) return sfail(UCN_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->loop_on) return UCN_OK;
  cudaError_t e = loop_kick(s);   // requests that wait get a launch to serve them
  __atomic_store_n(s->lstop_h, 1u, __ATOMIC_RELEASE);
  const cudaError_t w = cudaStreamSynchronize(s->loop_stream);   // the loop ends once the queue is empty
  if (e == cudaSuccess) e = w;
  loop_ended(s);
  if (e == cudaSuccess) e = s->loop_error;
  __atomic_store_n(s->lstop_h, 0u, __ATOMIC_RELEASE);
  s->loop_on = false;
  if (e != cudaSuccess) return sfail(UCN_ECUDA, "request loop failed: %s", cudaGetErrorString(e));
  // every published request has been delivered: the ring entries it wrote are complete
  for (int r = 0; r < s->R; ++r)
    if (s->ring_writing[r] && s->ring_lane[r] == LOOP_LANE) { s->ring_writing[r] = 0; s->ring_done[r] = 1; }
  return UCN_OK;
}

int ucn_serve_loop_capacity(ucn_server* s) {
  set_error_message("");
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  int cap = 0;
  const cudaError_t e = loop_launch(s, true, &cap);
  if (e != cudaSuccess) {
    sfail(UCN_EINVAL, "request loop: %s", cudaGetErrorString(e));
    return -1;
  }
  return cap;
}

int ucn_serve_loop_launches(ucn_server* s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  return s->loop_launches;
}

int ucn_serve_free_slots(ucn_server* s) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  retire_ended(s);
  int n = 0;
  for (int v : s->slot_state) n += (v == SLOT_FREE);
  return n;
}

}  // extern "C"
