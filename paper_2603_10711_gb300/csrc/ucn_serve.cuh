// Serving internals shared by the host-driven launches (ucn_serve.cu) and the
// device-resident request loop (serve_loop_kernel, instantiated per model and
// precision in the ucn_*_loop.cu units): the request record, the slot arrays,
// the per-request scatter and keep steps, and the loop itself.
#pragma once
#include "ucn_kernels.cuh"
#include "ucn_lanes.cuh"

namespace ucn {

// Offsets (in doubles) of one request record: slot, ring entry to read (warm
// start; -1: none), ring entry to fill (-1: none), the request's ticket (its
// delivery tag), horizon, obstacle count, the problem data of one instance,
// then the guesses.  Integers and bytes are stored as doubles (exact; tickets
// below 2^53).
struct RecLayout {
  int K, RING, RINGW, TAG, N, NOBS, DT, PRM, QD, XR, RD, UR, QND, QN, XLO, XHI, ULO, UHI, XI, XT, TM, OC, OR, SETS, XG, UG,
      END;
};
inline RecLayout rec_layout(int NX, int NU, int MO, int Xn, int Un) {
  RecLayout r;
  int o = 0;
  r.K = o++; r.RING = o++; r.RINGW = o++; r.TAG = o++; r.N = o++; r.NOBS = o++; r.DT = o++;
  r.PRM = o; o += 8;
  r.QD = o; o += NX; r.XR = o; o += NX; r.RD = o; o += NU; r.UR = o; o += NU;
  r.QND = o; o += NX; r.QN = o; o += NX; r.XLO = o; o += NX; r.XHI = o; o += NX;
  r.ULO = o; o += NU; r.UHI = o; o += NU; r.XI = o; o += NX; r.XT = o; o += NX; r.TM = o; o += NX;
  r.OC = o; o += 3 * MO; r.OR = o; o += MO; r.SETS = o; o += UCN_SET_PARAMS;
  r.XG = o; o += Xn * NX; r.UG = o; o += Un * NU;
  r.END = (o + 1) / 2 * 2;   // 16-byte records
  return r;
}

// The slot arrays and the ring of kept results (by value to the kernels).
struct ServeDev {
  int NX, NU, MO, Xn, Un, REC, RES;
  long long state_per_slot;
  RecLayout rl;
  int *N, *nobs;
  double *dt, *prm, *Qd, *xr, *Rd, *ur, *QNd, *qN, *xlo, *xhi, *ulo, *uhi, *xi, *xt, *oc, *orr, *sets;
  unsigned char *tm, *warm;
  unsigned long long* tag;
  double *x0, *u0, *xo, *uo, *state;
  ucn_scp_stats* stats;
  double *ring_x, *ring_u, *ring_state;
};

// Loads of a request record and of ring entries.  HOST: the record lives in
// mapped host memory that the host rewrites between requests, so it is read
// uncached; ring entries written by another SM of the same launch are read
// from L2.
template <bool HOST>
__device__ __forceinline__ double rec_ld(const double* p) {
  if constexpr (HOST) return __ldcv(p);
  else return *p;
}
template <bool HOST>
__device__ __forceinline__ double ring_ld(const double* p) {
  if constexpr (HOST) return __ldcg(p);
  else return *p;
}

// The request record r into its slot's arrays (the CTA's threads share the
// copies): problem data, and the guess -- or, for a warm start, the guess and
// the ADMM state from the ring entry of the request it names.  Returns the slot.
template <bool HOST>
__device__ __forceinline__ int serve_scatter_one(const ServeDev& D, const double* r) {
  const int t = threadIdx.x, nt = blockDim.x;
  const RecLayout& L = D.rl;
  const int k = (int)rec_ld<HOST>(r + L.K), ring = (int)rec_ld<HOST>(r + L.RING), N = (int)rec_ld<HOST>(r + L.N);
  const int NX = D.NX, NU = D.NU, MO = D.MO;
  if (t == 0) {
    D.tag[k] = (unsigned long long)rec_ld<HOST>(r + L.TAG);
    D.N[k] = N;
    D.nobs[k] = (int)rec_ld<HOST>(r + L.NOBS);
    D.dt[k] = rec_ld<HOST>(r + L.DT);
    D.warm[k] = ring >= 0 ? 1 : 0;
  }
  for (int e = t; e < 8; e += nt) {
    D.prm[k * 8 + e] = rec_ld<HOST>(r + L.PRM + e);
    D.sets[k * UCN_SET_PARAMS + e] = rec_ld<HOST>(r + L.SETS + e);
  }
  for (int e = t; e < NX; e += nt) {
    D.Qd[k * NX + e] = rec_ld<HOST>(r + L.QD + e); D.xr[k * NX + e] = rec_ld<HOST>(r + L.XR + e);
    D.QNd[k * NX + e] = rec_ld<HOST>(r + L.QND + e); D.qN[k * NX + e] = rec_ld<HOST>(r + L.QN + e);
    D.xlo[k * NX + e] = rec_ld<HOST>(r + L.XLO + e); D.xhi[k * NX + e] = rec_ld<HOST>(r + L.XHI + e);
    D.xi[k * NX + e] = rec_ld<HOST>(r + L.XI + e); D.xt[k * NX + e] = rec_ld<HOST>(r + L.XT + e);
    D.tm[k * NX + e] = (unsigned char)rec_ld<HOST>(r + L.TM + e);
  }
  for (int e = t; e < NU; e += nt) {
    D.Rd[k * NU + e] = rec_ld<HOST>(r + L.RD + e); D.ur[k * NU + e] = rec_ld<HOST>(r + L.UR + e);
    D.ulo[k * NU + e] = rec_ld<HOST>(r + L.ULO + e); D.uhi[k * NU + e] = rec_ld<HOST>(r + L.UHI + e);
  }
  for (int e = t; e < 3 * MO; e += nt) D.oc[(long long)k * 3 * MO + e] = rec_ld<HOST>(r + L.OC + e);
  for (int e = t; e < MO; e += nt) D.orr[(long long)k * MO + e] = rec_ld<HOST>(r + L.OR + e);
  double* x0 = D.x0 + (long long)k * D.Xn * NX;
  double* u0 = D.u0 + (long long)k * D.Un * NU;
  if (ring >= 0) {
    const double* rx = D.ring_x + (long long)ring * D.Xn * NX;
    const double* ru = D.ring_u + (long long)ring * D.Un * NU;
    const double* rs = D.ring_state + (long long)ring * D.state_per_slot;
    double* st = D.state + (long long)k * D.state_per_slot;
    for (int e = t; e < (N + 1) * NX; e += nt) x0[e] = ring_ld<HOST>(rx + e);
    for (int e = t; e < N * NU; e += nt) u0[e] = ring_ld<HOST>(ru + e);
    for (long long e = t; e < D.state_per_slot; e += nt) st[e] = ring_ld<HOST>(rs + e);
  } else {
    for (int e = t; e < (N + 1) * NX; e += nt) x0[e] = rec_ld<HOST>(r + L.XG + e);
    for (int e = t; e < N * NU; e += nt) u0[e] = rec_ld<HOST>(r + L.UG + e);
  }
  return k;
}

// The finished request of record r: its trajectory and final ADMM state into
// the ring entry assigned to it (warm starts of later requests).
template <bool HOST>
__device__ __forceinline__ void serve_keep_one(const ServeDev& D, const double* r) {
  const int t = threadIdx.x, nt = blockDim.x;
  const RecLayout& L = D.rl;
  const int k = (int)rec_ld<HOST>(r + L.K), ringw = (int)rec_ld<HOST>(r + L.RINGW), N = (int)rec_ld<HOST>(r + L.N);
  if (ringw < 0) return;
  const int NX = D.NX, NU = D.NU;
  const double* xo = D.xo + (long long)k * D.Xn * NX;
  const double* uo = D.uo + (long long)k * D.Un * NU;
  double* rx = D.ring_x + (long long)ringw * D.Xn * NX;
  double* ru = D.ring_u + (long long)ringw * D.Un * NU;
  double* rs = D.ring_state + (long long)ringw * D.state_per_slot;
  const double* st = D.state + (long long)k * D.state_per_slot;
  for (int e = t; e < (N + 1) * NX; e += nt) rx[e] = xo[e];
  for (int e = t; e < N * NU; e += nt) ru[e] = uo[e];
  for (long long e = t; e < D.state_per_slot; e += nt) rs[e] = st[e];
}

// ------------------------------------------------------------------ the device-resident request loop
// The host publishes request q by writing its slot's record, then
// queue[q % S] = slot, then head = q + 1 (release).  CTAs claim requests in
// order with a compare-and-swap on `next`, which never passes head.  The queue
// entry is read before the claim: a claim of q that succeeds means q was
// unclaimed while the entry was read, and while q and every later request is
// unclaimed each holds its own slot, so S + 1 of them cannot exist -- the entry
// still named q's slot.
struct LoopDev {
  const double* rec;               // per-slot request records [S][REC] (mapped host memory, device view)
  const long long* queue;          // slot of published request q at queue[q % S] (mapped)
  const unsigned long long* head;  // requests published (mapped; written by the host)
  const unsigned* stop;            // nonzero: end once every published request is claimed (mapped)
  unsigned long long* next;        // requests claimed so far (device memory; never reset)
  unsigned long long idle_ns;      // the loop ends once no request has been published for this long
  int S;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: the slot of the next request, or -1 when the loop should end (stop
// requested and nothing left to claim, or no request published to the server
// for Q.idle_ns).  The idle clock restarts whenever the head moves, whichever
// CTA claims the request, so that every CTA of the loop stays while requests
// keep arriving and all of them end together once the server has been quiet
// for the idle time.  Every wait is a bounded sleep.
__device__ __forceinline__ long long loop_claim(const LoopDev& Q, unsigned long long& idle_t0,
                                                unsigned long long& seen_head) {
  unsigned sleep_ns = 32;
  for (;;) {
    const unsigned long long h = ld_acquire_sys_u64(Q.head);
    if (h != seen_head) {
      seen_head = h;
      idle_t0 = globaltimer_ns();
    }
    unsigned long long n = *(volatile unsigned long long*)Q.next;
    while (n < h) {
      const long long k = *(volatile const long long*)(Q.queue + n % (unsigned long long)Q.S);
      const unsigned long long prev = atomicCAS(Q.next, n, n + 1);
      if (prev == n) return k;
      n = prev;
    }
    if (*(volatile const unsigned*)Q.stop) return -1;
    if (globaltimer_ns() - idle_t0 > Q.idle_ns) return -1;
    __nanosleep(sleep_ns);
    if (sleep_ns < 2048) sleep_ns *= 2;
  }
}

// One CTA of the loop: claim a request, scatter its record into its slot, run
// the fused SCP solve of that slot (one thread per node, or TPN = 4 lanes per
// node), keep its result in the ring, deliver it to host memory, repeat.  The
// solve itself is the launch-per-batch kernels' body with the instance index
// given, so the arithmetic is theirs.
template <class M, class T, bool SMEM, bool REFINE, int TPN>
__device__ __forceinline__ void serve_loop_body(const LoopDev& Q, const ServeDev& D, const ProblemDev& P,
                                                const Layout& L, int* status) {
  __shared__ long long slot;
  unsigned long long idle_t0 = globaltimer_ns(), seen_head = ~0ull;
  ProblemDev Ps = P;
  Ps.res_host = nullptr;   // the solve delivers nothing itself: the ring entry is written first
  for (;;) {
    if (threadIdx.x == 0) slot = loop_claim(Q, idle_t0, seen_head);
    __syncthreads();
    const long long k = slot;
    __syncthreads();
    if (k < 0) return;
    const double* r = Q.rec + k * (long long)D.REC;
    serve_scatter_one<true>(D, r);
    __syncthreads();
    if constexpr (TPN == 4)
      scp_lanes_body<M, T, SMEM, REFINE, false, 4>(Ps, L, D.x0, D.u0, D.xo, D.uo, D.stats, status, (int)k);
    else
      scp_body<M, T, SMEM, REFINE, false, true>(Ps, L, D.x0, D.u0, D.xo, D.uo, D.stats, status, (int)k);
    __syncthreads();
    serve_keep_one<true>(D, r);
    __threadfence();
    __syncthreads();
    deliver_result(P, (int)k, D.xo, D.uo, D.stats);
  }
}

template <class M, class T, bool SMEM, bool REFINE, int TPN>
__global__ void __launch_bounds__(TPN == 4 ? LANES_MAX_THREADS : MAX_THREADS)
    serve_loop_kernel(LoopDev Q, ServeDev D, ProblemDev P, Layout L, int* status) {
  serve_loop_body<M, T, SMEM, REFINE, TPN>(Q, D, P, L, status);
}

// Everything a loop launch needs besides the kernel choice.
struct LoopCfg {
  const LoopDev* Q;
  const ServeDev* D;
  const ProblemDev* P;
  const Layout* L;
  int* status;
  bool smem;
  long long smem_bytes;
  int threads;      // CTA size
  int tpn;          // 1, or 4 (lane kernel, quadrotor)
  int ctas;         // CTAs to launch (0: every CTA that can be resident)
  cudaStream_t stream;
  int* launched_ctas = nullptr;   // out: CTAs launched (or that could be resident, with query)
  bool query = false;             // only report how many CTAs can be resident at once
};

template <class M, class T, bool SMEM, bool R, int TPN>
cudaError_t launch_loop_v(const LoopCfg& c) {
  auto k = serve_loop_kernel<M, T, SMEM, R, TPN>;
  cudaError_t e = cudaSuccess;
  if (SMEM) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_bytes);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, c.threads, SMEM ? c.smem_bytes : 0);
  if (e != cudaSuccess) return e;
  // more CTAs than can be resident would only start as resident ones end
  const int cap = sms * per_sm;
  if (c.query) {
    if (c.launched_ctas) *c.launched_ctas = cap;
    return cudaSuccess;
  }
  if (cap < 1) return cudaErrorInvalidConfiguration;
  const int n = c.ctas > 0 ? (c.ctas < cap ? c.ctas : cap) : cap;
  k<<<n, c.threads, SMEM ? c.smem_bytes : 0, c.stream>>>(*c.Q, *c.D, *c.P, *c.L, c.status);
  e = cudaGetLastError();
  if (e == cudaSuccess && c.launched_ctas) *c.launched_ctas = n;
  return e;
}

template <class M, class T, bool R>
cudaError_t launch_loop_t(const LoopCfg& c) {
  if constexpr (LaneModel<M>::value) {
    if (c.tpn == 4) return c.smem ? launch_loop_v<M, T, true, R, 4>(c) : launch_loop_v<M, T, false, R, 4>(c);
  }
  if (c.tpn != 1) return cudaErrorInvalidConfiguration;
  return c.smem ? launch_loop_v<M, T, true, R, 1>(c) : launch_loop_v<M, T, false, R, 1>(c);
}

}  // namespace ucn

// The loop launcher of one model and precision.
#define UCN_DEFINE_LOOP_LAUNCHER(NAME, MODEL, T, REFINE)                                                   \
  namespace ucn {                                                                                          \
  cudaError_t NAME##_loop(const LoopCfg& c) { return launch_loop_t<MODEL, T, REFINE>(c); }                 \
  }

// One loop variant (records in shared memory or the global workspace; threads
// per node) in its own translation unit.
#define UCN_LOOP_V(MODEL, T, SMEM, REFINE, TPN) cudaError_t ucn::launch_loop_v<ucn::MODEL, T, SMEM, REFINE, TPN>(const ucn::LoopCfg&)
#define UCN_INSTANTIATE_LOOP(MODEL, T, SMEM, REFINE, TPN) template UCN_LOOP_V(MODEL, T, SMEM, REFINE, TPN);
#define UCN_EXTERN_LOOP(MODEL, T, SMEM, REFINE, TPN) extern template UCN_LOOP_V(MODEL, T, SMEM, REFINE, TPN);
