// Device path of SCP + consensus ADMM (arXiv 2603.10711) for sm_103a.
//
// Mapping.  One CTA owns one instance; thread i owns time node i (state x_i,
// control u_i, and its consensus copies).  Per-node data live in a
// structure-of-arrays block (element k of node i at base[off + k*S + i]) in
// shared memory when the instance fits, else in a per-instance global
// workspace slice; the same code serves both.  The only inter-node exchange
// of an ADMM iteration is nearest-neighbour (Eq. (5) needs A_{i-1}x_{i-1}+...
// from the left; Step 1 needs mu_{i+1} + rho_dyn z_{i+1} from the right),
// done through two shared exchange vectors and two CTA barriers.
//
// Coordinates.  The QP of Eq. (2) is solved in deviations from the nominal,
// delta = x - xbar.  Every ADMM step of Sec. III-B commutes with that
// translation (the duals are unchanged), so the iterates are the paper's up to
// rounding; the affine term becomes c_i = RK4(xbar_i, ubar_i) - xbar_{i+1},
// which is small, and that is what lets the FP32 path keep its accuracy.
#pragma once
#include <type_traits>

#include "ucn_math.cuh"

namespace ucn {

enum { ST_OK = 0, ST_NUMERIC = 4, ST_NOTCONV = 5, ST_TIMEOUT = 6 };
constexpr int MAX_THREADS = 256;   // CTA size cap: horizons up to 255 nodes

struct ProblemDev {
  int model, nx, nu, batch, max_obs;
  const int* N;
  const long long* xoff;
  const long long* uoff;
  const long long* soff;
  const double *dt, *params, *Qd, *xref, *Rd, *uref, *QNd, *qN;
  const double *xlo, *xhi, *ulo, *uhi, *xinit, *xtarget;
  const unsigned char* tmask;
  const int* nobs;
  const double *obs_c, *obs_r, *sets;
  double rho_eq, rho_dyn, rho_geo, rho_final;
  int scp_iters, admm_iters, stop;
  double tr_init, tr_min, tr_max, w_d, defect_tol, step_tol;
  unsigned long long timeout_ns;
  double* state_abs;       // exported ADMM state, absolute FP64 (soff layout)
  char* ws;                // per-instance node storage when it does not fit in shared memory
  const int* order;        // CTA -> instance map of the fused solve (NULL: identity)
  int group;               // scenarios per group (<= 1: independent instances)
  const double* rho_fac;   // penalty factor of each SCP iteration (NULL: computed in the kernel)
  int gclusters;           // thread-block clusters per group (group = gclusters x cluster size)
  double* gx;              // exchange slots of the scenarios [instance][2][16]
  unsigned* gflag;         // per instance: last exchange published (+1); zeroed per launch
  unsigned long long gwait_ns;   // bound on a wait for another scenario of the group
  const unsigned char* warm;     // per instance: 1 = start from the ADMM state in state_abs (NULL: all cold)
  // Result delivery to mapped host memory (serving; NULL: none): at its end each
  // CTA copies its instance's stats (16 doubles), x and u into res_host[b]
  // (res_stride doubles per instance), then sets res_flag[b] = res_tag[b].
  double* res_host;
  unsigned long long* res_flag;
  const unsigned long long* res_tag;
  long long res_stride;
};

static_assert(sizeof(ucn_scp_stats) == 16 * sizeof(double), "a result record starts with 16 doubles of stats");

// The end of a fused solve with result delivery: every thread copies its share
// of the instance's x and u (just written to xout, uout by this CTA) into the
// mapped host record and fences them system-wide, then one thread copies the
// stats record, fences, and publishes the instance's tag in its flag -- the
// host sees the flag only after the record.  No thread waits on the host.
__device__ __forceinline__ void deliver_result(const ProblemDev& P, int b, const double* xout, const double* uout,
                                               const ucn_scp_stats* stats) {
  if (!P.res_host) return;
  const int N = P.N[b], nx = P.nx, nu = P.nu;
  const long long xo = P.xoff[b], uo = P.uoff[b];
  double* r = P.res_host + (long long)b * P.res_stride;
  for (int e = threadIdx.x; e < (N + 1) * nx; e += blockDim.x) r[16 + e] = xout[xo * nx + e];
  for (int e = threadIdx.x; e < N * nu; e += blockDim.x) r[16 + (N + 1) * nx + e] = uout[uo * nu + e];
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* sd = reinterpret_cast<const double*>(stats + b);
    for (int e = 0; e < 16; ++e) r[e] = sd[e];
    __threadfence_system();
    *(volatile unsigned long long*)(P.res_flag + b) = P.res_tag[b];
  }
}

// Fixed part of a node record: compile-time element offsets of every per-node
// array.  The mirror arrays (whose length depends on the obstacle count) follow
// at the runtime offsets Layout::oS / oNus / oMd, then the matrices A, B, H^-1
// at Layout::oA / oB / oH -- absent from the record when they live in registers.
template <class M>
struct Rec {
  static constexpr int NX = M::NX, NU = M::NU, NN = NX + NU;
  static constexpr int C = 0;
  static constexpr int Xlo = C + NX, Xhi = Xlo + NX, Ulo = Xhi + NX, Uhi = Ulo + NU;
  static constexpr int X = Uhi + NU, Z = X + NX, Lam = Z + NX, Mu = Lam + NX, Xh = Mu + NX, Nux = Xh + NX;
  static constexpr int U = Nux + NX, Uh = U + NU, Nuu = Uh + NU, Ex1 = Nuu + NU, Ex2 = Ex1 + NX, END = Ex2 + NX;
  // wide record (FP64, or double-float on the FP32 path): nominal state,
  // nominal control, candidate state (exchange)
  static constexpr int Xbar = 0, Ubar = NX, Xc = NX + NU, DEND = 2 * NX + NU;
};

// Per-instance constants of the FP32 path in double-float, converted from the
// problem's FP64 arrays once per launch, so that the per-SCP-iteration setup,
// rollout and cost read no FP64 value: bounds, references, boundary states,
// cost weights, model parameters and the RK4 step h, h/2, h/6.
template <class M>
struct CB {
  static constexpr int NX = M::NX, NU = M::NU;
  static constexpr int Xlo = 0, Xhi = NX, Xref = 2 * NX, Xinit = 3 * NX, Xtgt = 4 * NX, Qd = 5 * NX, QNd = 6 * NX,
                       QN = 7 * NX, Ulo = 8 * NX, Uhi = Ulo + NU, Uref = Uhi + NU, Rd = Uref + NU, Prm = Rd + NU,
                       Step = Prm + 8, END = Step + 3;
};

// Where the per-node records of one instance live.
//  shared memory: node i's record at t + i*NS (NS odd: conflict-free banks),
//                 FP64 record at d + i*DS (DS odd);
//  global slice:  element k of node i at t[k*S + i] (coalesced SoA).
struct Layout {
  int S, NS, DS;           // SoA stride (nodes); AoS record strides (elements)
  int MS, MD, MB;          // mirror scalars / mirror data per node; exported mirror blocks
  int oS, oNus, oMd;       // runtime offsets of the mirror arrays in the record
  int oA, oB, oH;          // matrices in the record (-1 when register-resident)
  long long tbytes;        // bytes of the T region (16-byte multiple)
  long long bytes;         // bytes per instance
  long long oC;            // byte offset of the CB block (FP32 path; -1 without)
  long long oPH;           // byte offset of the pair kernel's per-lane H^-1 records (-1 without)
};

// Per-thread view of its node.  W is the wide type of the precision (FP64,
// or double-float for the FP32 path).
template <class T, bool AOS>
struct Node {
  typedef typename WideOf<T>::type W;
  T* t;          // T region base
  W* d;          // wide region base
  W* c;          // CB block of the instance (FP32 path)
  int S, NS, DS, i, N;
  __device__ __forceinline__ T& at(int off, int k) const { return AOS ? t[i * NS + off + k] : t[(long long)(off + k) * S + i]; }
  __device__ __forceinline__ T& nb(int off, int k, int j) const { return AOS ? t[j * NS + off + k] : t[(long long)(off + k) * S + j]; }
  __device__ __forceinline__ W& dat(int off, int k) const { return AOS ? d[i * DS + off + k] : d[(long long)(off + k) * S + i]; }
  __device__ __forceinline__ W& dnb(int off, int k, int j) const { return AOS ? d[j * DS + off + k] : d[(long long)(off + k) * S + j]; }
};

// The wide path of a compute type is double-float (FP32 path).
template <class T> struct IsDF { static constexpr bool value = std::is_same<typename WideOf<T>::type, DF>::value; };

// Models whose mirror sets are the linearised obstacles (the quadrotors); the
// others carry the Mars sets (thrust ball and lower bound, glide-slope cone).
template <class M> struct IsQuad {
  static constexpr bool value = std::is_same<M, Quad12>::value || std::is_same<M, Quat13>::value;
};
// The 6-DOF Mars model: its own sets (glide slope on r, tilt on (qy, qz), body
// rate ball, thrust ball and lower bound, gimbal cone on the body thrust).
template <class M> struct IsMars14 { static constexpr bool value = std::is_same<M, Mars14>::value; };
// Mirror slots of the 6-DOF model in the record (scalars s and nu_s; data).
struct M14 {
  static constexpr int S_CONE = 0, S_BALL = 3, S_HALF = 6, S_TILT = 7, S_W = 9, S_GIM = 12, MS = 15;
  static constexpr int D_N = 0, D_BD = 3, D_R = 4, D_U = 7, D_Q = 10, D_W = 12, MD = 15;
};
// Models the lane kernel serves (rows split evenly over 4 lanes).
template <class M> struct LaneModel {
  static constexpr bool value = IsQuad<M>::value && M::NX % 4 == 0 && M::NU % 4 == 0;
};

// Storage of a node's matrices A_i, B_i and the packed H_i^-1.  Small models
// keep them in registers (every index below is a compile-time constant after
// unrolling), which takes ~60% of the shared-memory traffic out of the ADMM
// iteration; larger ones keep them in the node record.
// Record entries per linearised obstacle (normal, bound): padded to 5 in FP32
// so that the lanes of the lane kernel, which take every fourth obstacle, fall
// in distinct banks.
template <class T> struct ObsStride { static constexpr int value = sizeof(T) == 4 ? 5 : 4; };

// Row strides of A and B in the record: odd (NX | 1, NU | 1) for the FP32 lane
// layout, so that lanes reading different rows, or different columns, of their
// node's matrix fall in distinct banks; unpadded otherwise.
template <class M, class T> struct MatStride {
  static constexpr bool pad = LaneModel<M>::value && sizeof(T) == 4;
  static constexpr int A = pad ? (M::NX | 1) : M::NX, B = pad ? (M::NU | 1) : M::NU;
};
// Which entries of A_i = dRK4/dx are exactly zero (0) or exactly one (1) at
// every nominal, else 2.  Forward-mode differentiation gives an exact 0 where
// the dynamics do not couple two states and an exact 1 where a state enters
// its own update only additively.  3-DOF Mars (x = r, v, m; r' = v,
// v' = T/m + g, m' = -alpha |T|): r_{k+1} depends on r (identity), on v along
// the same axis and on m; v_{k+1} on v (identity) and m; m_{k+1} on m alone.
template <class M> struct APattern {
  __host__ __device__ static constexpr int kind(int, int) { return 2; }
};
template <> struct APattern<Mars7> {
  __host__ __device__ static constexpr int kind(int r, int c) {
    return r == c ? 1 : (r < 3 && c == r + 3) ? 2 : (r < 6 && c == 6) ? 2 : 0;
  }
};

template <class M, class T, bool AOS>
struct SmemMats {
  __host__ __device__ static constexpr int akind(int, int) { return 2; }
  Node<T, AOS> nd;
  int oA, oB, oH;
  __device__ __forceinline__ T& A(int r, int c) const { return nd.at(oA, r * MatStride<M, T>::A + c); }
  __device__ __forceinline__ T& B(int r, int c) const { return nd.at(oB, r * MatStride<M, T>::B + c); }
  __device__ __forceinline__ T& H(int k) const { return nd.at(oH, k); }
};
template <class M, class T>
struct RegMats {
  __host__ __device__ static constexpr int akind(int, int) { return 2; }
  static constexpr int NN = M::NX + M::NU;
  mutable T a[M::NX * M::NX], b[M::NX * M::NU], h[NN * (NN + 1) / 2];
  __device__ __forceinline__ T& A(int r, int c) const { return a[r * M::NX + c]; }
  __device__ __forceinline__ T& B(int r, int c) const { return b[r * M::NU + c]; }
  __device__ __forceinline__ T& H(int k) const { return h[k]; }
};
template <class M> struct SmallModel {
  static constexpr int NN = M::NX + M::NU;
  static constexpr bool value = M::NX * M::NX + M::NX * M::NU + NN * (NN + 1) / 2 <= 128;
};
// Register-resident matrices of the kernel's own Jacobians: the products skip
// the structural zeros of A_i and add its exact ones (APattern) -- the same
// sums up to rounding (an exact one's term is added without a multiply, which
// the compiler may fuse with that term's own product: bitwise equal in FP64,
// within a few float ulps in FP32), fewer instructions, and no registers for
// those entries.  The 3-DOF Mars model keeps 9 of its 49 entries.
template <class M, class T>
struct RegMatsS : RegMats<M, T> {
  __host__ __device__ static constexpr int akind(int r, int c) { return APattern<M>::kind(r, c); }
};
// OWNJ: the matrices are the kernel's own Jacobians (their structure holds);
// a caller's A (ucn_admm_solve) is taken as dense.
template <class M, class T, bool AOS, bool OWNJ = false>
using MatsFor = typename std::conditional<AOS && SmallModel<M>::value,
                                          typename std::conditional<OWNJ, RegMatsS<M, T>, RegMats<M, T>>::type,
                                          SmemMats<M, T, AOS>>::type;

// acc += A(r, c) v, and acc += A(k, r) A(k, c), with the storage's structure of
// A: exact zeros skipped, exact ones added without the product.
template <class MS, class T>
__device__ __forceinline__ void acc_A(T& acc, const MS& MT, int r, int c, T v) {
  if (MS::akind(r, c) == 1) acc += v;
  else if (MS::akind(r, c) == 2) acc += MT.A(r, c) * v;
}
template <class MS, class T>
__device__ __forceinline__ void acc_AA(T& acc, const MS& MT, int k, int r, int c) {
  const int kr = MS::akind(k, r), kc = MS::akind(k, c);
  if (kr == 0 || kc == 0) return;
  if (kr == 1 && kc == 1) acc += T(1);
  else if (kr == 1) acc += MT.A(k, c);
  else if (kc == 1) acc += MT.A(k, r);
  else acc += MT.A(k, r) * MT.A(k, c);
}

template <class M, class T, bool AOS>
__device__ __forceinline__ void init_mats(SmemMats<M, T, AOS>& m, const Node<T, AOS>& nd, const Layout& L) {
  m.nd = nd; m.oA = L.oA; m.oB = L.oB; m.oH = L.oH;
}
template <class M, class T, bool AOS>
__device__ __forceinline__ void init_mats(RegMats<M, T>& m, const Node<T, AOS>& nd, const Layout& L) {}

// Per-node constants of one SCP iteration, held in registers across the ADMM
// loop: the cost gradient (q_i, r_i) in deviations and the diagonal of H_i
// without its A/B and mirror Gram terms.
template <class M, class T>
struct NodeConst {
  T q[M::NX + M::NU];
  T hd[M::NX + M::NU];
};

// Per-instance constants read once per kernel into registers, so that the
// ADMM loop touches no global memory and no FP64 arithmetic.
template <class T>
struct Inst {
  int nobs;                 // quadrotor: obstacles of this instance
  bool cone, ball, half;    // Mars: glide-slope cone, thrust ball, thrust lower bound
  T tau, tmax, ca, sa;      // cone tan(half-angle) and its cos/sin; thrust ball radius
  bool gim, tilt, wball;    // Mars 6-DOF: gimbal cone, tilt ball, body-rate ball
  T tg, cg, sg, rtilt, wmax;
  bool run_cost, term_quad; // nonzero running weights / terminal quadratic weights
  T prm[8];                 // model constants in T (Jacobian passes)
};

// Obstacles of instance b, clamped to [0, max_obs]: ucn_problem_create checks
// the counts on the host, but the no-allocation entry point reads them from a
// caller's device array it cannot check, and a count beyond max_obs would
// index past the instance's obstacle and mirror slots.
__device__ __forceinline__ int nobs_of(const ProblemDev& P, int b) {
  const int v = P.nobs[b];
  return v < 0 ? 0 : (v > P.max_obs ? P.max_obs : v);
}

// A value the compiler cannot trace back to how it was computed.  The set
// flags below come from FP64 comparisons; left traceable, the compiler may
// recompute such a flag by its FP64 comparison at every branch on it instead
// of keeping it (measured on GB300: ten FP64-pipe instructions per ADMM
// iteration, on a pipe that runs at 1/64 of the FP32 rate there).
__device__ __forceinline__ unsigned opaque_u32(unsigned v) {
  asm volatile("mov.b32 %0, %0;" : "+r"(v));
  return v;
}

template <class M, class T>
__device__ __forceinline__ Inst<T> make_inst(const ProblemDev& P, int b) {
  Inst<T> I;
  I.nobs = IsQuad<M>::value ? nobs_of(P, b) : 0;
  const double tmin = IsQuad<M>::value ? 0.0 : P.sets[b * UCN_SET_PARAMS + 0];
  const double tmax = IsQuad<M>::value ? 0.0 : P.sets[b * UCN_SET_PARAMS + 1];
  const double tau = IsQuad<M>::value ? 0.0 : P.sets[b * UCN_SET_PARAMS + 2];
  I.tau = (T)tau; I.tmax = (T)tmax;
  const double ca = 1.0 / sqrt(1.0 + tau * tau);
  I.ca = (T)ca; I.sa = (T)(tau * ca);
  const double tg = IsMars14<M>::value ? P.sets[b * UCN_SET_PARAMS + 3] : 0.0;
  const double rt = IsMars14<M>::value ? P.sets[b * UCN_SET_PARAMS + 4] : 0.0;
  const double wm = IsMars14<M>::value ? P.sets[b * UCN_SET_PARAMS + 5] : 0.0;
  const double cg = 1.0 / sqrt(1.0 + tg * tg);
  I.tg = (T)tg; I.cg = (T)cg; I.sg = (T)(tg * cg); I.rtilt = (T)rt; I.wmax = (T)wm;
  bool rc = false, tq = false;
  for (int j = 0; j < M::NX; ++j) { rc = rc || P.Qd[b * M::NX + j] != 0.0; tq = tq || P.QNd[b * M::NX + j] != 0.0; }
  for (int j = 0; j < M::NU; ++j) rc = rc || P.Rd[b * M::NU + j] != 0.0;
  const unsigned f = opaque_u32((tmin > 0.0 ? 1u : 0u) | (tmax > 0.0 ? 2u : 0u) | (tau > 0.0 ? 4u : 0u) |
                                (tg > 0.0 ? 8u : 0u) | (rt > 0.0 ? 16u : 0u) | (wm > 0.0 ? 32u : 0u) |
                                (rc ? 64u : 0u) | (tq ? 128u : 0u));
  I.half = f & 1u; I.ball = f & 2u; I.cone = f & 4u;
  I.gim = f & 8u; I.tilt = f & 16u; I.wball = f & 32u;
  I.run_cost = f & 64u; I.term_quad = f & 128u;
  for (int k = 0; k < 8; ++k) I.prm[k] = (T)P.params[b * 8 + k];
  return I;
}

// Per-instance scalars in shared memory.
struct InstShared {
  unsigned long long xbar[2];   // split barrier of the ADMM exchange + failure flag
  double red[32][6];
  double Jn, radius;
  double rho[3];            // rho_eq, rho_dyn, rho_geo of the SCP iteration
  float rhof[3];            // the same in FP32 (no conversion per thread)
  double out[8];
  int fail;
  int accept, stop, status;
};

// Per-CTA state of a scenario group's exchanges (one CTA per scenario).
struct GroupShared {
  double mine[2][16];   // this CTA's contribution to the current exchange (double-buffered)
  double u0[4];         // the consensus u-hat_0 of the latest iteration, absolute
  int gfail;            // sticky: a wait for another scenario of the group gave up
};

// Sequence state of the group exchanges, identical in every thread of the group.
struct GroupX {
  unsigned epoch;       // exchanges done
  int g, k;             // group index, scenario index within the group
  unsigned long long* bar;   // the CTA's split barrier (mbarrier) and its failure flag
  unsigned ph;               // completed phases of the split barrier
};

// Split CTA barrier on an mbarrier object in shared memory: every thread
// arrives once per phase (release), may do independent work, then waits for
// the phase to complete (acquire).  The wait is bounded; a wait that gives up
// sets bar[1] (reported as a numerical failure) and returns.
__device__ __forceinline__ void split_barrier_init(unsigned long long* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
  bar[1] = 0ull;
}
__device__ __forceinline__ void split_barrier_arrive(unsigned long long* bar) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(a) : "memory");
}
__device__ __forceinline__ void split_barrier_wait(unsigned long long* bar, unsigned& ph) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  const unsigned parity = ph & 1u;
  ++ph;
  for (int it = 0; it < (1 << 20); ++it) {
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return;
  }
  bar[1] = 1ull;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// All-reduce over a scenario group of the NV values that warp 0 of every CTA
// has put in G->mine[X.epoch & 1]: entries [0, ns) summed, the rest maxed.
// Every thread of every CTA of the group calls it the same number of times;
// thread 0 receives the result in out, and every CTA of the group the same
// bits (the same operations on the same data).  Two forms, each the faster one
// measured in its regime:
//
// One cluster per group (group <= 16): one cluster barrier, then lane r of
// warp 0 loads rank r's values through distributed shared memory (all loads
// in flight at once) and a butterfly over the warp combines them.
template <int NV>
__device__ void group_allreduce_cluster(GroupShared* G, GroupX& X, int ns, double* out) {
  const int par = X.epoch & 1;
  cluster_sync();
  if (threadIdx.x < 32) {
    const unsigned lane = threadIdx.x, nk = cluster_size();
    double pv[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) pv[j] = j < ns ? 0.0 : -INFINITY;
    if (lane < nk) {
#pragma unroll
      for (int j = 0; j < NV; ++j) pv[j] = ld_cluster(&G->mine[par][j], lane);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const double t = __shfl_xor_sync(0xffffffffu, pv[j], o);
        pv[j] = j < ns ? pv[j] + t : fmax(pv[j], t);
      }
    if (lane == 0)
      for (int j = 0; j < NV; ++j) out[j] = pv[j];
  }
  X.epoch++;
}

// Several clusters per group: no barrier at all; lane 0 publishes the CTA's
// values to its global slot and releases its counter; lane r then waits
// (relaxed polling, then acquire; time-bounded) for scenario r's counter (r,
// r+32, ...), loads that scenario's values, and a butterfly over the warp
// combines them.  Slots are double-buffered by the exchange's parity: a
// scenario can be at most one exchange ahead of another.  A wait that gives up
// marks the group failed and stops waiting for the rest of the launch (status
// ETIMEOUT), so the kernel always ends.
template <int NV>
__device__ void group_allreduce_flat(const ProblemDev& P, GroupShared* G, GroupX& X, int ns, double* out) {
  static_assert(NV <= 16, "exchange slots hold 16 values");
  const int par = X.epoch & 1;
  if (threadIdx.x < 32) {
    __syncwarp();
    const int lane = threadIdx.x, K = P.group;
    const long long base = (long long)X.g * K;
    if (lane == 0) {
      double* slot = P.gx + ((base + X.k) * 2 + par) * 16;
      for (int j = 0; j < NV; ++j) slot[j] = G->mine[par][j];
      st_release_gpu(&P.gflag[base + X.k], X.epoch + 1);
    }
    double pv[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) pv[j] = j < ns ? 0.0 : -INFINITY;
    for (int r = lane; r < K; r += 32) {
      const unsigned* f = &P.gflag[base + r];
      bool ok = !G->gfail;
      if (ok) {
        // relaxed polling, one acquire once the counter is seen (an acquire per
        // poll would also cost the SM its L1 lines); the clock is read every
        // 256 polls
        unsigned long long t0 = 0;
        for (unsigned spins = 1; ld_relaxed_gpu(f) < X.epoch + 1; ++spins) {
          if ((spins & 255u) == 0u) {
            const unsigned long long now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > P.gwait_ns) { ok = false; G->gfail = 1; break; }
          }
        }
        if (ok) (void)ld_acquire_gpu(f);
      }
      if (!ok) continue;
      const double* src = P.gx + ((base + r) * 2 + par) * 16;
      double v[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) v[j] = __ldcg(src + j);
#pragma unroll
      for (int j = 0; j < NV; ++j) pv[j] = j < ns ? pv[j] + v[j] : fmax(pv[j], v[j]);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const double t = __shfl_xor_sync(0xffffffffu, pv[j], o);
        pv[j] = j < ns ? pv[j] + t : fmax(pv[j], t);
      }
    if (lane == 0)
      for (int j = 0; j < NV; ++j) out[j] = pv[j];
  }
  X.epoch++;
}

template <int NV>
__device__ __forceinline__ void group_allreduce(const ProblemDev& P, GroupShared* G, GroupX& X, int ns, double* out) {
  if (P.gclusters <= 1) group_allreduce_cluster<NV>(G, X, ns, out);
  else group_allreduce_flat<NV>(P, G, X, ns, out);
}

// The end of a group kernel: no CTA of a one-cluster group may exit while
// another can still read its shared memory.
__device__ __forceinline__ void group_finish(const ProblemDev& P) {
  if (P.gclusters <= 1) cluster_sync();
}

// The exchange area exists in the shared memory of group kernels only.
template <bool GROUP>
__device__ __forceinline__ GroupShared* group_slot() {
  if constexpr (GROUP) {
    __shared__ GroupShared g;
    return &g;
  } else {
    return nullptr;
  }
}

template <class T> __device__ __forceinline__ T rho_of(const InstShared& sh, int r) { return (T)sh.rho[r]; }
template <> __device__ __forceinline__ float rho_of<float>(const InstShared& sh, int r) { return sh.rhof[r]; }

// ------------------------------------------------------------------ block reduction
// Reduces up to 6 FP64 values: entries [0, nsum) summed, [nsum, nval) maxed.
__device__ __forceinline__ void block_reduce(InstShared& sh, double* v, int nsum, int nval) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < nval; ++k) v[k] = (k < nsum) ? warp_sum(v[k]) : warp_max(v[k]);
  if (lane == 0)
    for (int k = 0; k < nval; ++k) sh.red[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < nval; ++k) {
      double a = (lane < nw) ? sh.red[lane][k] : (k < nsum ? 0.0 : -1.0);
      a = (k < nsum) ? warp_sum(a) : warp_max(a);
      if (lane == 0) sh.out[k] = a;
    }
  }
  __syncthreads();
  for (int k = 0; k < nval; ++k) v[k] = sh.out[k];
  __syncthreads();
}

// The same over double-float sums s[0, ns) and float maxima m[0, nm) (ns + nm
// <= 6), with no FP64 instruction outside warp 0's final conversion; every
// thread receives the sums then the maxima, as doubles, in out[0, ns + nm).
// The double-float sum is commutative bit for bit (its error terms are exact),
// so every lane of a butterfly holds the same bits.
__device__ __forceinline__ DF df_shfl_xor(DF a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ void block_reduce_df(InstShared& sh, DF* s, int ns, float* m, int nm, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  DF* red = reinterpret_cast<DF*>(&sh.red[0][0]);
  float* redf = reinterpret_cast<float*>(&sh.red[0][0]);
  for (int o = 16; o > 0; o >>= 1) {
    for (int k = 0; k < ns; ++k) s[k] = df_add(s[k], df_shfl_xor(s[k], o));
    for (int k = 0; k < nm; ++k) m[k] = fmaxf(m[k], __shfl_xor_sync(0xffffffffu, m[k], o));
  }
  if (lane == 0) {
    for (int k = 0; k < ns; ++k) red[warp * 6 + k] = s[k];
    for (int k = 0; k < nm; ++k) redf[2 * (warp * 6 + ns + k)] = m[k];
  }
  __syncthreads();
  if (warp == 0) {
    DF a[6];
    float b[6];
    for (int k = 0; k < ns; ++k) a[k] = (lane < nw) ? red[lane * 6 + k] : DF();
    for (int k = 0; k < nm; ++k) b[k] = (lane < nw) ? redf[2 * (lane * 6 + ns + k)] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) {
      for (int k = 0; k < ns; ++k) a[k] = df_add(a[k], df_shfl_xor(a[k], o));
      for (int k = 0; k < nm; ++k) b[k] = fmaxf(b[k], __shfl_xor_sync(0xffffffffu, b[k], o));
    }
    if (lane == 0) {
      for (int k = 0; k < ns; ++k) sh.out[k] = df_to_double(a[k]);
      for (int k = 0; k < nm; ++k) sh.out[ns + k] = (double)b[k];
    }
  }
  __syncthreads();
  for (int k = 0; k < ns + nm; ++k) out[k] = sh.out[k];
  __syncthreads();
}

// CTA totals of the squared residual norms, as doubles in res[0..1].
__device__ __forceinline__ void reduce_residuals(InstShared& sh, double rp, double rdl, double* res) {
  double v[2] = {rp, rdl};
  block_reduce(sh, v, 2, 2);
  res[0] = v[0];
  res[1] = v[1];
}
__device__ __forceinline__ void reduce_residuals(InstShared& sh, DF rp, DF rdl, double* res) {
  DF s2[2] = {rp, rdl};
  block_reduce_df(sh, s2, 2, nullptr, 0, res);
}

// ------------------------------------------------------------------ per-node pieces
// The CB block of the instance (FP32 path): every thread of the CTA converts
// a share of the entries; the caller synchronises before the first use.
template <class M, class T, bool AOS>
__device__ void stage_consts(const Node<T, AOS>& nd, const ProblemDev& P, int b) {
  if constexpr (IsDF<T>::value) {
    typedef CB<M> C;
    constexpr int NX = M::NX, NU = M::NU;
    for (int e = threadIdx.x; e < C::END; e += blockDim.x) {
      double v;
      if (e < C::Xhi) v = P.xlo[b * NX + e - C::Xlo];
      else if (e < C::Xref) v = P.xhi[b * NX + e - C::Xhi];
      else if (e < C::Xinit) v = P.xref[b * NX + e - C::Xref];
      else if (e < C::Xtgt) v = P.xinit[b * NX + e - C::Xinit];
      else if (e < C::Qd) v = P.xtarget[b * NX + e - C::Xtgt];
      else if (e < C::QNd) v = P.Qd[b * NX + e - C::Qd];
      else if (e < C::QN) v = P.QNd[b * NX + e - C::QNd];
      else if (e < C::Ulo) v = P.qN[b * NX + e - C::QN];
      else if (e < C::Uhi) v = P.ulo[b * NU + e - C::Ulo];
      else if (e < C::Uref) v = P.uhi[b * NU + e - C::Uhi];
      else if (e < C::Rd) v = P.uref[b * NU + e - C::Uref];
      else if (e < C::Prm) v = P.Rd[b * NU + e - C::Rd];
      else if (e < C::Step) v = P.params[b * 8 + e - C::Prm];
      else v = P.dt[b] * (e == C::Step ? 1.0 : e == C::Step + 1 ? 0.5 : 1.0 / 6.0);
      nd.c[e] = df_from(v);
    }
  }
}

// Nominal of node i from packed global trajectories.
template <class M, class T, bool AOS>
__device__ void load_nominal(const Node<T, AOS>& nd, const Layout& L, const double* xg, const double* ug,
                             long long xo, long long uo) {
  typedef typename Node<T, AOS>::W W;
  for (int j = 0; j < M::NX; ++j) nd.dat(Rec<M>::Xbar, j) = wide_from_double<W>(xg[(xo + nd.i) * M::NX + j]);
  if (nd.i < nd.N)
    for (int j = 0; j < M::NU; ++j) nd.dat(Rec<M>::Ubar, j) = wide_from_double<W>(ug[(uo + nd.i) * M::NU + j]);
}

template <class M, class T, bool AOS>
__device__ __forceinline__ void read_nominal(const Node<T, AOS>& nd, bool hasU, typename Node<T, AOS>::W* xb,
                                             typename Node<T, AOS>::W* ub) {
  typedef typename Node<T, AOS>::W W;
#pragma unroll
  for (int j = 0; j < M::NX; ++j) xb[j] = nd.dat(Rec<M>::Xbar, j);
#pragma unroll
  for (int j = 0; j < M::NU; ++j) ub[j] = hasU ? nd.dat(Rec<M>::Ubar, j) : W();
}

// One RK4 step of the instance's model in the wide type: FP64 from the problem
// arrays, or double-float from the CB block.
template <class M, class T, bool AOS>
__device__ __forceinline__ void rk4_wide(const Node<T, AOS>& nd, const ProblemDev& P, int b,
                                         const typename Node<T, AOS>::W* x, const typename Node<T, AOS>::W* u,
                                         typename Node<T, AOS>::W* xn) {
  if constexpr (IsDF<T>::value) {
    typedef CB<M> C;
    rk4h<M, DF, DF, DF>(nd.c + C::Prm, nd.c[C::Step], nd.c[C::Step + 1], nd.c[C::Step + 2], x, u, xn);
  } else {
    rk4<M, double>(P.params + b * 8, P.dt[b], x, u, xn);
  }
}

// |a| of a wide value, as a double for the FP64 path and rounded to float for
// double-float (maxima and tolerance tests need no more).
__device__ __forceinline__ double wide_abs_round(double a) { return fabs(a); }
__device__ __forceinline__ float wide_abs_round(DF a) { return fabsf(df_to_float(a)); }
__device__ __forceinline__ double wide_abs(double a) { return fabs(a); }
__device__ __forceinline__ DF wide_abs(DF a) { return a.hi < 0.0f ? df_neg(a) : a; }

// A_i, B_i by forward-mode differentiation of the RK4 map (Eq. (2b)), in T.
template <class M, class T, bool AOS, class MS>
__device__ __forceinline__ void node_jacobians(const Node<T, AOS>& nd, const MS& MT, const T* prm, const Step3<T>& hs) {
  constexpr int NX = M::NX, NU = M::NU;
  typename Node<T, AOS>::W xb[NX], ub[NU];
  read_nominal<M, T, AOS>(nd, true, xb, ub);
  T xt[NX], ut[NU];
#pragma unroll
  for (int j = 0; j < NX; ++j) xt[j] = wide_to<T>(xb[j]);
#pragma unroll
  for (int j = 0; j < NU; ++j) ut[j] = wide_to<T>(ub[j]);
  if constexpr (std::is_same<M, Mars7>::value && std::is_same<MS, RegMatsS<M, T>>::value) {
    // The structure of A (APattern<Mars7>), whose products read nothing else: the r
    // columns are unit vectors, and a v_i column holds besides its unit entry
    // d r_i / d v_i, which the RK4 weights of r' = v make h/6 (1 + 2 + 2 + 1) for every
    // axis and nominal (the value a forward-mode pass along v_i computes, bit for bit).
    // One pass along m and the thrust gives the rest: the m column of A, and B.
    T cols[4][NX];
    if constexpr (std::is_same<T, float>::value) {
      rk4_jvpn<M, T, 4>(prm, hs, xt, ut, NX - 1, 1, cols);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) rk4_jvp<M, T>(prm, hs, xt, ut, NX - 1 + q, cols[q]);
    }
    const T dh = hs.h6 * T(6);
#pragma unroll
    for (int r = 0; r < 3; ++r) MT.A(r, 3 + r) = dh;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      MT.A(r, NX - 1) = cols[0][r];
#pragma unroll
      for (int c = 0; c < NU; ++c) MT.B(r, c) = cols[1 + c][r];
    }
  } else if constexpr (std::is_same<T, float>::value) {
    // FP32: five columns per pass (the value of the RK4 map once for the five),
    // the remainder one column per pass
    constexpr int KD = 5;
#pragma unroll
    for (int dir = 0; dir < NX + NU; dir += KD) {
      if (dir + KD <= NX + NU) {
        T cols[KD][NX];
        rk4_jvpn<M, T, KD>(prm, hs, xt, ut, dir, 1, cols);
#pragma unroll
        for (int q = 0; q < KD; ++q)
#pragma unroll
          for (int r = 0; r < NX; ++r) {
            if (dir + q < NX) MT.A(r, dir + q) = cols[q][r];
            else MT.B(r, dir + q - NX) = cols[q][r];
          }
      } else {
#pragma unroll
        for (int d1 = dir; d1 < NX + NU; ++d1) {
          T col[NX];
          rk4_jvp<M, T>(prm, hs, xt, ut, d1, col);
#pragma unroll
          for (int r = 0; r < NX; ++r) {
            if (d1 < NX) MT.A(r, d1) = col[r];
            else MT.B(r, d1 - NX) = col[r];
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int dir = 0; dir < NX + NU; ++dir) {
      T col[NX];
      rk4_jvp<M, T>(prm, hs, xt, ut, dir, col);
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        if (dir < NX) MT.A(r, dir) = col[r];
        else MT.B(r, dir - NX) = col[r];
      }
    }
  }
}

// QP data of node i at the nominal: cost gradient in deviations, the
// trust-region boxes of Eq. (2c) (with the boundary conditions of Eq. (1c)
// as degenerate boxes at nodes 0 and N), and the mirror-set data.
template <class M, class T, bool AOS>
__device__ void node_setup(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, const Inst<T>& I, int b,
                           double radius, T re, T rg, NodeConst<M, T>& K) {
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  typename Node<T, AOS>::W xb[NX], ub[NU];
  read_nominal<M, T, AOS>(nd, i < N, xb, ub);
  const bool term = (i == N);
  if constexpr (IsDF<T>::value) {
    // the same quantities from the CB block in double-float, rounded to T
    typedef CB<M> C;
    const DF* cb = nd.c;
    const T rad = (T)radius;
    // running nodes of a problem without running state cost (the Mars batch):
    // zero gradient and weight without the double-float product
    const bool cost = term || I.run_cost;
    for (int j = 0; j < NX; ++j) {
      const DF w = term ? cb[C::QNd + j] : cb[C::Qd + j];
      if (cost) {
        DF gq = df_mul(df_sub(xb[j], cb[C::Xref + j]), w);
        if (term) gq = df_add(gq, cb[C::QN + j]);
        K.q[j] = df_to_float(gq);
      } else {
        K.q[j] = T(0);
      }
      K.hd[j] = df_to_float(w) + rg + (i > 0 ? re : T(0));
      T lo = fmaxf(wide_diff<T>(cb[C::Xlo + j], xb[j]), -rad);
      T hi = fminf(wide_diff<T>(cb[C::Xhi + j], xb[j]), rad);
      if (i == 0) lo = hi = wide_diff<T>(cb[C::Xinit + j], xb[j]);
      else if (term && P.tmask[b * NX + j]) lo = hi = wide_diff<T>(cb[C::Xtgt + j], xb[j]);
      nd.at(Rec<M>::Xlo, j) = lo;
      nd.at(Rec<M>::Xhi, j) = hi;
    }
    for (int j = 0; j < NU; ++j) { K.q[NX + j] = T(0); K.hd[NX + j] = T(1); }
    if (!term) {
      for (int j = 0; j < NU; ++j) {
        const DF w = cb[C::Rd + j];
        K.q[NX + j] = I.run_cost ? df_to_float(df_mul(df_sub(ub[j], cb[C::Uref + j]), w)) : T(0);
        K.hd[NX + j] = df_to_float(w) + rg;
        nd.at(Rec<M>::Ulo, j) = fmaxf(wide_diff<T>(cb[C::Ulo + j], ub[j]), -rad);
        nd.at(Rec<M>::Uhi, j) = fminf(wide_diff<T>(cb[C::Uhi + j], ub[j]), rad);
      }
    }
  } else {
  for (int j = 0; j < NX; ++j) {
    const double w = term ? P.QNd[b * NX + j] : P.Qd[b * NX + j];
    K.q[j] = (T)(w * (xb[j] - P.xref[b * NX + j]) + (term ? P.qN[b * NX + j] : 0.0));
    K.hd[j] = (T)w + rg + (i > 0 ? re : T(0));
    double lo = fmax(P.xlo[b * NX + j], xb[j] - radius) - xb[j];
    double hi = fmin(P.xhi[b * NX + j], xb[j] + radius) - xb[j];
    if (i == 0) lo = hi = P.xinit[b * NX + j] - xb[j];
    else if (term && P.tmask[b * NX + j]) lo = hi = P.xtarget[b * NX + j] - xb[j];
    nd.at(Rec<M>::Xlo, j) = (T)lo;
    nd.at(Rec<M>::Xhi, j) = (T)hi;
  }
  for (int j = 0; j < NU; ++j) { K.q[NX + j] = T(0); K.hd[NX + j] = T(1); }
  if (!term) {
    for (int j = 0; j < NU; ++j) {
      K.q[NX + j] = (T)(P.Rd[b * NU + j] * (ub[j] - P.uref[b * NU + j]));
      K.hd[NX + j] = (T)P.Rd[b * NU + j] + rg;
      nd.at(Rec<M>::Ulo, j) = (T)(fmax(P.ulo[b * NU + j], ub[j] - radius) - ub[j]);
      nd.at(Rec<M>::Uhi, j) = (T)(fmin(P.uhi[b * NU + j], ub[j] + radius) - ub[j]);
    }
  }
  }
  if constexpr (IsQuad<M>::value) {
    // Obstacle j linearised about the nominal position: n = (p - c)/|p - c|,
    // keep n^T p >= n^T c + r; in deviations n^T dp >= n^T (c - pbar) + r.
    const int no = nobs_of(P, b);
    for (int j = 0; j < no; ++j) {
      const double* c = &P.obs_c[((long long)b * P.max_obs + j) * 3];
      // offset from the centre in T (|p - c| is of the order of the radius: no cancellation)
      const T dp[3] = {wide_to<T>(xb[0]) - (T)c[0], wide_to<T>(xb[1]) - (T)c[1], wide_to<T>(xb[2]) - (T)c[2]};
      T nv[3] = {dp[0], dp[1], dp[2]};
      T nn = sqrt_(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      if (nn < T(1e-12)) { nv[0] = 0; nv[1] = 0; nv[2] = 1; nn = 1; }
      const T inn = T(1) / nn;
      const T n0 = nv[0] * inn, n1 = nv[1] * inn, n2 = nv[2] * inn;
      const T bd = -(n0 * dp[0] + n1 * dp[1] + n2 * dp[2]) + (T)P.obs_r[(long long)b * P.max_obs + j];
      nd.at(L.oMd, ObsStride<T>::value * j + 0) = (T)n0;
      nd.at(L.oMd, ObsStride<T>::value * j + 1) = (T)n1;
      nd.at(L.oMd, ObsStride<T>::value * j + 2) = (T)n2;
      nd.at(L.oMd, ObsStride<T>::value * j + 3) = (T)bd;
    }
  } else {
    // nominal position / thrust in T, the offsets of the cone and ball projections
    constexpr int RC = IsMars14<M>::value ? 1 : 0;   // position's first state
    for (int k = 0; k < 3; ++k) nd.at(L.oMd, 4 + k) = wide_to<T>(xb[RC + k]);
    for (int k = 0; k < 3; ++k) nd.at(L.oMd, 7 + k) = wide_to<T>(ub[k]);
    if constexpr (IsMars14<M>::value) {   // nominal (qy, qz) and body rates
      for (int k = 0; k < 2; ++k) nd.at(L.oMd, M14::D_Q + k) = wide_to<T>(xb[9 + k]);
      for (int k = 0; k < 3; ++k) nd.at(L.oMd, M14::D_W + k) = wide_to<T>(xb[11 + k]);
    }
    // Thrust lower bound |T| >= Tmin linearised: nbar^T T >= Tmin, nbar = Tbar/|Tbar|.
    if (!term) {
      const T ut[3] = {wide_to<T>(ub[0]), wide_to<T>(ub[1]), wide_to<T>(ub[2])};
      T nv[3] = {ut[0], ut[1], ut[2]};
      T nn = sqrt_(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      if (nn < T(1e-12)) { nv[0] = 1; nv[1] = 0; nv[2] = 0; nn = 1; }
      const T inn = T(1) / nn;
      const T n0 = nv[0] * inn, n1 = nv[1] * inn, n2 = nv[2] * inn;
      nd.at(L.oMd, 0) = n0;
      nd.at(L.oMd, 1) = n1;
      nd.at(L.oMd, 2) = n2;
      nd.at(L.oMd, 3) = (T)P.sets[b * UCN_SET_PARAMS + 0] - (n0 * ut[0] + n1 * ut[1] + n2 * ut[2]);
    }
  }
}

// Packed lower-triangular index (row r, column c <= r).
__host__ __device__ constexpr int pk(int r, int c) { return r * (r + 1) / 2 + c; }

template <class T, int n, class MS>
__device__ __forceinline__ bool factor_invert_packed(const MS& MT);

// H_i of Eq. (4) plus rho_geo G_j^T G_j for each mirror set, assembled in
// packed form and factored H = L L^T in place (unpivoted Cholesky; the
// diagonal holds 1/L_jj).  Returns false on a non-positive pivot.  Node N,
// which has no control, is factored at the same size with an identity
// control block and no coupling, so its state block is H_N exactly.
template <class M, class T, bool AOS, int n, class MS>
__device__ __forceinline__ bool node_factor(const Node<T, AOS>& nd, const MS& MT, const Layout& L, const Inst<T>& I,
                                            const NodeConst<M, T>& K, T rd, T rg) {
  constexpr int NX = M::NX;
  const int i = nd.i, N = nd.N;
  const bool hasU = (n > NX);
  const bool term = (i == N);
  #pragma unroll
  for (int r = 0; r < n; ++r) {
    #pragma unroll
    for (int c = 0; c <= r; ++c) {
      T h = T(0);
      if (r < NX) {  // H11
        if (r == c) h = K.hd[r];
        if (!term) {
          T acc = T(0);
          #pragma unroll
          for (int k = 0; k < NX; ++k) acc_AA(acc, MT, k, r, c);
          h += rd * acc;
        }
        if constexpr (IsQuad<M>::value) {
          if (r < 3 && c < 3) {
            T acc = T(0);
            #pragma unroll
            for (int j = 0; j < I.nobs; ++j) acc += nd.at(L.oMd, ObsStride<T>::value * j + r) * nd.at(L.oMd, ObsStride<T>::value * j + c);
            h += rg * acc;
          }
        } else {
          constexpr int RC = IsMars14<M>::value ? 1 : 0;
          if (r >= RC && r < RC + 3 && r == c && I.cone) h += rg;
          if constexpr (IsMars14<M>::value) {
            if (r == c && I.tilt && (r == 9 || r == 10)) h += rg;
            if (r == c && I.wball && r >= 11 && r <= 13) h += rg;
          }
        }
      } else if (c < NX) {  // H21 = H12^T (zero at node N: no control there)
        T acc = T(0);
        #pragma unroll
        for (int k = 0; k < NX; ++k) acc_A(acc, MT, k, c, MT.B(k, r - NX));
        h = term ? T(0) : rd * acc;
      } else {  // H22 (identity at node N, decoupled from the state block)
        const int rr = r - NX, cc = c - NX;
        if (rr == cc) h = K.hd[r];
        T acc = T(0);
        #pragma unroll
        for (int k = 0; k < NX; ++k) acc += MT.B(k, rr) * MT.B(k, cc);
        if (!term) h += rd * acc;
        if constexpr (!IsQuad<M>::value) {
          if (rr < 3 && cc < 3 && !term) {
            if (rr == cc && I.ball) h += rg;
            if (I.half) h += rg * nd.at(L.oMd, rr) * nd.at(L.oMd, cc);
            if constexpr (IsMars14<M>::value) {
              if (rr == cc && I.gim) h += rg;
            }
          }
        }
      }
      MT.H(pk(r, c)) = h;
    }
  }
  (void)hasU;
  return factor_invert_packed<T, n>(MT);
}

// Packed H (lower triangle) -> packed H^-1 in place: unpivoted Cholesky
// H = L L^T, then L^-1 and H^-1 = L^-T L^-1.  Returns false on a non-positive
// pivot (replaced by 1 so that the arithmetic stays finite).
template <class T, int n, class MS>
__device__ __forceinline__ bool factor_invert_packed(const MS& MT) {
  bool ok = true;
  #pragma unroll
  for (int j = 0; j < n; ++j) {
    T s = MT.H(pk(j, j));
    #pragma unroll
    for (int k = 0; k < j; ++k) { const T l = MT.H(pk(j, k)); s -= l * l; }
    if (!(s > T(0))) { ok = false; s = T(1); }
    const T inv = inv_sqrt_(s);
    MT.H(pk(j, j)) = inv;
    #pragma unroll
    for (int r = j + 1; r < n; ++r) {
      T t = MT.H(pk(r, j));
      #pragma unroll
      for (int k = 0; k < j; ++k) t -= MT.H(pk(r, k)) * MT.H(pk(j, k));
      MT.H(pk(r, j)) = t * inv;
    }
  }
  // In place: L -> L^-1 (column by column; the diagonal already holds 1/L_jj),
  // then L^-1 -> H^-1 = L^-T L^-1 (row by row, lower triangle).  The ADMM
  // loop then solves H xi = g by one symmetric mat-vec: the same solve as the
  // forward/back substitution, with independent dot products instead of a
  // chain of n dependent steps.
  #pragma unroll
  for (int j = 0; j < n; ++j) {
    T col[n];
    col[j] = MT.H(pk(j, j));
    #pragma unroll
    for (int r = j + 1; r < n; ++r) {
      T t = T(0);
      #pragma unroll
      for (int k = j; k < r; ++k) t += MT.H(pk(r, k)) * (k == j ? col[j] : col[k]);
      col[r] = -t * MT.H(pk(r, r));
    }
    #pragma unroll
    for (int r = j + 1; r < n; ++r) MT.H(pk(r, j)) = col[r];
  }
  #pragma unroll
  for (int r = 0; r < n; ++r) {
    T row[n];
    #pragma unroll
    for (int c = 0; c <= r; ++c) {
      T t = T(0);
      #pragma unroll
      for (int k = r; k < n; ++k) t += MT.H(pk(k, r)) * MT.H(pk(k, c));
      row[c] = t;
    }
    #pragma unroll
    for (int c = 0; c <= r; ++c) MT.H(pk(r, c)) = row[c];
  }
  return ok;
}

// xi = H^-1 g with the cached packed inverse (lower triangle of a symmetric matrix).
template <class T, int n, class MS>
__device__ __forceinline__ void sym_solve(const MS& MT, const T* g, T* xi) {
#pragma unroll
  for (int r = 0; r < n; ++r) {
    T t = T(0);
#pragma unroll
    for (int c = 0; c < n; ++c) t += MT.H(r >= c ? pk(r, c) : pk(c, r)) * g[c];
    xi[r] = t;
  }
}

// H xi without forming H (A, B, the cost diagonals, the rho terms and the
// mirror Gram terms), for the refinement residual g - H xi.
template <class M, class T, bool AOS, int n, class MS>
__device__ __forceinline__ void apply_H(const Node<T, AOS>& nd, const MS& MT, const Layout& L, const Inst<T>& I,
                                        const NodeConst<M, T>& K, T rd, T rg, const T* xi, T* out) {
  constexpr int NX = M::NX, NU = M::NU;
#pragma unroll
  for (int j = 0; j < NX; ++j) out[j] = K.hd[j] * xi[j];
  const bool coupled = nd.i < nd.N;   // node N: identity control block, no coupling
  if constexpr (n > NX) {
   if (!coupled) {
#pragma unroll
    for (int j = 0; j < NU; ++j) out[NX + j] = K.hd[NX + j] * xi[NX + j];
   } else {
    T v[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NX; ++c) acc_A(acc, MT, r, c, xi[c]);
#pragma unroll
      for (int c = 0; c < NU; ++c) acc += MT.B(r, c) * xi[NX + c];
      v[r] = rd * acc;
    }
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) acc_A(acc, MT, k, j, v[k]);
      out[j] += acc;
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) acc += MT.B(k, j) * v[k];
      out[NX + j] = K.hd[NX + j] * xi[NX + j] + acc;
    }
   }
  }
  if constexpr (IsQuad<M>::value) {
    for (int j = 0; j < I.nobs; ++j) {
      const T n0 = nd.at(L.oMd, ObsStride<T>::value * j), n1 = nd.at(L.oMd, ObsStride<T>::value * j + 1), n2 = nd.at(L.oMd, ObsStride<T>::value * j + 2);
      const T y = rg * (n0 * xi[0] + n1 * xi[1] + n2 * xi[2]);
      out[0] += n0 * y; out[1] += n1 * y; out[2] += n2 * y;
    }
  } else {
    constexpr int RC = IsMars14<M>::value ? 1 : 0;
    if (I.cone) { out[RC] += rg * xi[RC]; out[RC + 1] += rg * xi[RC + 1]; out[RC + 2] += rg * xi[RC + 2]; }
    if constexpr (IsMars14<M>::value) {
      if (I.tilt) { out[9] += rg * xi[9]; out[10] += rg * xi[10]; }
      if (I.wball) { out[11] += rg * xi[11]; out[12] += rg * xi[12]; out[13] += rg * xi[13]; }
    }
    if (n > NX && coupled) {
      if (I.ball) { out[NX] += rg * xi[NX]; out[NX + 1] += rg * xi[NX + 1]; out[NX + 2] += rg * xi[NX + 2]; }
      if constexpr (IsMars14<M>::value) {
        if (I.gim) { out[NX] += rg * xi[NX]; out[NX + 1] += rg * xi[NX + 1]; out[NX + 2] += rg * xi[NX + 2]; }
      }
      if (I.half) {
        const T n0 = nd.at(L.oMd, 0), n1 = nd.at(L.oMd, 1), n2 = nd.at(L.oMd, 2);
        const T y = rg * (n0 * xi[NX] + n1 * xi[NX + 1] + n2 * xi[NX + 2]);
        out[NX] += n0 * y; out[NX + 1] += n1 * y; out[NX + 2] += n2 * y;
      }
    }
  }
}

// The node's own ADMM variables z, lambda, mu, nu_x, nu_u (no other node reads
// them).  REG: held in registers for the length of an ADMM call, loaded from
// the node record before it and written back after it (the register-resident
// FP32 kernels of small models, where the structure of A leaves room);
// otherwise references into the record.
template <class M, class T, bool AOS, bool REG>
struct NodeState;
template <class M, class T, bool AOS>
struct NodeState<M, T, AOS, true> {
  mutable T zv[M::NX], lamv[M::NX], muv[M::NX], nuxv[M::NX], nuuv[M::NU];
  __device__ __forceinline__ T& z(int j) const { return zv[j]; }
  __device__ __forceinline__ T& lam(int j) const { return lamv[j]; }
  __device__ __forceinline__ T& mu(int j) const { return muv[j]; }
  __device__ __forceinline__ T& nux(int j) const { return nuxv[j]; }
  __device__ __forceinline__ T& nuu(int j) const { return nuuv[j]; }
  __device__ __forceinline__ void load(const Node<T, AOS>& nd) {
#pragma unroll
    for (int j = 0; j < M::NX; ++j) {
      zv[j] = nd.at(Rec<M>::Z, j); lamv[j] = nd.at(Rec<M>::Lam, j); muv[j] = nd.at(Rec<M>::Mu, j);
      nuxv[j] = nd.at(Rec<M>::Nux, j);
    }
#pragma unroll
    for (int j = 0; j < M::NU; ++j) nuuv[j] = nd.at(Rec<M>::Nuu, j);
  }
  __device__ __forceinline__ void store(const Node<T, AOS>& nd) const {
#pragma unroll
    for (int j = 0; j < M::NX; ++j) {
      nd.at(Rec<M>::Z, j) = zv[j]; nd.at(Rec<M>::Lam, j) = lamv[j]; nd.at(Rec<M>::Mu, j) = muv[j];
      nd.at(Rec<M>::Nux, j) = nuxv[j];
    }
#pragma unroll
    for (int j = 0; j < M::NU; ++j) nd.at(Rec<M>::Nuu, j) = nuuv[j];
  }
};
template <class M, class T, bool AOS>
struct NodeState<M, T, AOS, false> {
  Node<T, AOS> nd;
  __device__ __forceinline__ T& z(int j) const { return nd.at(Rec<M>::Z, j); }
  __device__ __forceinline__ T& lam(int j) const { return nd.at(Rec<M>::Lam, j); }
  __device__ __forceinline__ T& mu(int j) const { return nd.at(Rec<M>::Mu, j); }
  __device__ __forceinline__ T& nux(int j) const { return nd.at(Rec<M>::Nux, j); }
  __device__ __forceinline__ T& nuu(int j) const { return nd.at(Rec<M>::Nuu, j); }
  __device__ __forceinline__ void load(const Node<T, AOS>& n) { nd = n; }
  __device__ __forceinline__ void store(const Node<T, AOS>&) const {}
};
// REGS: the kernel variant leaves registers for the state (the 3-CTAs-per-SM
// variant of the one-thread kernel does not).
template <class M, class T, bool AOS, bool REGS = true>
using NodeStateFor = NodeState<M, T, AOS, REGS && AOS && SmallModel<M>::value && std::is_same<T, float>::value>;

// Right-hand side g_i of Step 1 (stationarity of Eq. (3) in (x_i, u_i)).
template <class M, class T, bool AOS, int n, class MS, class NS>
__device__ __forceinline__ void node_rhs(const Node<T, AOS>& nd, const MS& MT, const Layout& L, const Inst<T>& I,
                                         const NodeConst<M, T>& K, const NS& S, T re, T rd, T rg, T* g) {
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i;
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    T v = -K.q[j] + rg * nd.at(Rec<M>::Xh, j) - S.nux(j);
    if (i > 0) v += re * S.z(j) - S.lam(j);
    g[j] = v;
  }
  if constexpr (n > NX) {
   if (i < nd.N) {
    // w_i = mu_{i+1} + rho_dyn (z_{i+1} - c_i); node i+1 publishes mu + rho_dyn z
    T w[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) w[k] = nd.nb(Rec<M>::Ex2, k, i + 1) - rd * nd.at(Rec<M>::C, k);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) acc_A(acc, MT, k, j, w[k]);
      g[j] += acc;
    }
#pragma unroll
    for (int j = 0; j < NU; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) acc += MT.B(k, j) * w[k];
      g[NX + j] = -K.q[NX + j] + acc + rg * nd.at(Rec<M>::Uh, j) - S.nuu(j);
    }
   } else {
#pragma unroll
    for (int j = 0; j < NU; ++j) g[NX + j] = T(0);   // node N: no control
   }
  }
  if constexpr (IsQuad<M>::value) {
    for (int j = 0; j < I.nobs; ++j) {
      const T a = rg * nd.at(L.oS, j) - nd.at(L.oNus, j);
      g[0] += nd.at(L.oMd, ObsStride<T>::value * j) * a;
      g[1] += nd.at(L.oMd, ObsStride<T>::value * j + 1) * a;
      g[2] += nd.at(L.oMd, ObsStride<T>::value * j + 2) * a;
    }
  } else {
    constexpr int RC = IsMars14<M>::value ? 1 : 0;
    if (I.cone)
      for (int k = 0; k < 3; ++k) g[RC + k] += rg * nd.at(L.oS, k) - nd.at(L.oNus, k);
    if constexpr (IsMars14<M>::value) {
      if (I.tilt)
        for (int k = 0; k < 2; ++k) g[9 + k] += rg * nd.at(L.oS, M14::S_TILT + k) - nd.at(L.oNus, M14::S_TILT + k);
      if (I.wball)
        for (int k = 0; k < 3; ++k) g[11 + k] += rg * nd.at(L.oS, M14::S_W + k) - nd.at(L.oNus, M14::S_W + k);
    }
    if (n > NX && i < nd.N) {
      if constexpr (IsMars14<M>::value) {
        if (I.gim)
          for (int k = 0; k < 3; ++k) g[NX + k] += rg * nd.at(L.oS, M14::S_GIM + k) - nd.at(L.oNus, M14::S_GIM + k);
      }
      if (I.ball)
        for (int k = 0; k < 3; ++k) g[NX + k] += rg * nd.at(L.oS, 3 + k) - nd.at(L.oNus, 3 + k);
      if (I.half) {
        const T a = rg * nd.at(L.oS, 6) - nd.at(L.oNus, 6);
        for (int k = 0; k < 3; ++k) g[NX + k] += nd.at(L.oMd, k) * a;
      }
    }
  }
}

// Mirror projections (Step 3) and their dual ascent (Step 4) for the non-box
// sets; `sv` accumulates rho_geo G^T (s_new - s_old) for the dual residual,
// `rp` the squared primal residual |G xi - s|^2.  Initialisation (reseed)
// mode projects G xi alone and leaves the duals untouched.
template <class M, class T, bool AOS, int n>
__device__ __forceinline__ void node_mirrors(const Node<T, AOS>& nd, const Layout& L, const Inst<T>& I,
                                             T rg, T irg, const T* xi, bool reseed, bool want_res, T* sv, typename WideOf<T>::type& rp) {
  constexpr int NX = M::NX;
  if constexpr (IsQuad<M>::value) {
    for (int j = 0; j < I.nobs; ++j) {
      const T n0 = nd.at(L.oMd, ObsStride<T>::value * j), n1 = nd.at(L.oMd, ObsStride<T>::value * j + 1), n2 = nd.at(L.oMd, ObsStride<T>::value * j + 2);
      const T bd = nd.at(L.oMd, ObsStride<T>::value * j + 3);
      const T y = n0 * xi[0] + n1 * xi[1] + n2 * xi[2];
      if (reseed) { nd.at(L.oS, j) = maxv(bd, y); continue; }
      const T so = nd.at(L.oS, j);
      const T s = maxv(bd, y + nd.at(L.oNus, j) * irg);
      nd.at(L.oS, j) = s;
      nd.at(L.oNus, j) += rg * (y - s);
      if (want_res) {
        const T ds = rg * (s - so);
        sv[0] += n0 * ds; sv[1] += n1 * ds; sv[2] += n2 * ds;
        acc_sq_diff(rp, y, s);
      }
    }
  } else {
    T xb[3], ub[3];
    for (int k = 0; k < 3; ++k) xb[k] = nd.at(L.oMd, 4 + k);
    for (int k = 0; k < 3; ++k) ub[k] = (n > NX) ? nd.at(L.oMd, 7 + k) : T(0);
    constexpr int RC = IsMars14<M>::value ? 1 : 0;   // position's first state
    if (I.cone) {  // glide-slope cone on the position (t = Up)
      T v[3];
      for (int k = 0; k < 3; ++k) v[k] = xb[k] + xi[RC + k] + (reseed ? T(0) : nd.at(L.oNus, k) * irg);
      proj_cone3c(v, I.tau, I.ca, I.sa);
      for (int k = 0; k < 3; ++k) {
        const T s = v[k] - xb[k];
        if (reseed) { nd.at(L.oS, k) = s; continue; }
        const T so = nd.at(L.oS, k);
        nd.at(L.oS, k) = s;
        nd.at(L.oNus, k) += rg * (xi[RC + k] - s);
        if (want_res) { sv[RC + k] += rg * (s - so); acc_sq_diff(rp, xi[RC + k], s); }
      }
    }
    if constexpr (IsMars14<M>::value) {
      if (I.tilt) {  // |(qy, qz)| <= sin(theta_max / 2)
        T v[3];
        for (int k = 0; k < 2; ++k)
          v[k] = nd.at(L.oMd, M14::D_Q + k) + xi[9 + k] + (reseed ? T(0) : nd.at(L.oNus, M14::S_TILT + k) * irg);
        v[2] = T(0);
        proj_ball3(v, I.rtilt);
        for (int k = 0; k < 2; ++k) {
          const T s = v[k] - nd.at(L.oMd, M14::D_Q + k);
          if (reseed) { nd.at(L.oS, M14::S_TILT + k) = s; continue; }
          const T so = nd.at(L.oS, M14::S_TILT + k);
          nd.at(L.oS, M14::S_TILT + k) = s;
          nd.at(L.oNus, M14::S_TILT + k) += rg * (xi[9 + k] - s);
          if (want_res) { sv[9 + k] += rg * (s - so); acc_sq_diff(rp, xi[9 + k], s); }
        }
      }
      if (I.wball) {  // |omega| <= omega_max
        T v[3];
        for (int k = 0; k < 3; ++k)
          v[k] = nd.at(L.oMd, M14::D_W + k) + xi[11 + k] + (reseed ? T(0) : nd.at(L.oNus, M14::S_W + k) * irg);
        proj_ball3(v, I.wmax);
        for (int k = 0; k < 3; ++k) {
          const T s = v[k] - nd.at(L.oMd, M14::D_W + k);
          if (reseed) { nd.at(L.oS, M14::S_W + k) = s; continue; }
          const T so = nd.at(L.oS, M14::S_W + k);
          nd.at(L.oS, M14::S_W + k) = s;
          nd.at(L.oNus, M14::S_W + k) += rg * (xi[11 + k] - s);
          if (want_res) { sv[11 + k] += rg * (s - so); acc_sq_diff(rp, xi[11 + k], s); }
        }
      }
      if (n > NX && nd.i < nd.N) {
        if (I.gim) {  // gimbal: |(T_y, T_z)| <= tan(delta_max) T_x (t = body x)
          T v[3];
          for (int k = 0; k < 3; ++k) v[k] = ub[k] + xi[NX + k] + (reseed ? T(0) : nd.at(L.oNus, M14::S_GIM + k) * irg);
          proj_cone3c(v, I.tg, I.cg, I.sg);
          for (int k = 0; k < 3; ++k) {
            const T s = v[k] - ub[k];
            if (reseed) { nd.at(L.oS, M14::S_GIM + k) = s; continue; }
            const T so = nd.at(L.oS, M14::S_GIM + k);
            nd.at(L.oS, M14::S_GIM + k) = s;
            nd.at(L.oNus, M14::S_GIM + k) += rg * (xi[NX + k] - s);
            if (want_res) { sv[NX + k] += rg * (s - so); acc_sq_diff(rp, xi[NX + k], s); }
          }
        }
      }
    }
    if (n > NX && nd.i < nd.N) {   // control sets (node N has no control)
      if (I.ball) {  // |T| <= Tmax
        T v[3];
        for (int k = 0; k < 3; ++k) v[k] = ub[k] + xi[NX + k] + (reseed ? T(0) : nd.at(L.oNus, 3 + k) * irg);
        proj_ball3(v, I.tmax);
        for (int k = 0; k < 3; ++k) {
          const T s = v[k] - ub[k];
          if (reseed) { nd.at(L.oS, 3 + k) = s; continue; }
          const T so = nd.at(L.oS, 3 + k);
          nd.at(L.oS, 3 + k) = s;
          nd.at(L.oNus, 3 + k) += rg * (xi[NX + k] - s);
          if (want_res) { sv[NX + k] += rg * (s - so); acc_sq_diff(rp, xi[NX + k], s); }
        }
      }
      if (I.half) {  // linearised |T| >= Tmin
        const T n0 = nd.at(L.oMd, 0), n1 = nd.at(L.oMd, 1), n2 = nd.at(L.oMd, 2), bd = nd.at(L.oMd, 3);
        const T y = n0 * xi[NX] + n1 * xi[NX + 1] + n2 * xi[NX + 2];
        if (reseed) {
          nd.at(L.oS, 6) = maxv(bd, y);
        } else {
          const T so = nd.at(L.oS, 6);
          const T s = maxv(bd, y + nd.at(L.oNus, 6) * irg);
          nd.at(L.oS, 6) = s;
          nd.at(L.oNus, 6) += rg * (y - s);
          if (want_res) {
            const T ds = rg * (s - so);
            sv[NX] += n0 * ds; sv[NX + 1] += n1 * ds; sv[NX + 2] += n2 * ds;
            acc_sq_diff(rp, y, s);
          }
        }
      }
    }
  }
}

// Mirror initialisation / re-seeding from (x-hat, u-hat) in deviations.
template <class M, class T, bool AOS>
__device__ void node_reseed(const Node<T, AOS>& nd, const Layout& L, const Inst<T>& I) {
  constexpr int NX = M::NX, NU = M::NU;
  T xi[NX + NU], sv[NX + NU];
  typename WideOf<T>::type rp{};
  for (int j = 0; j < NX; ++j) xi[j] = nd.at(Rec<M>::Xh, j);
  if (nd.i < nd.N) {
    for (int j = 0; j < NU; ++j) xi[NX + j] = nd.at(Rec<M>::Uh, j);
    node_mirrors<M, T, AOS, NX + NU>(nd, L, I, T(1), T(1), xi, true, false, sv, rp);
  } else {
    node_mirrors<M, T, AOS, NX>(nd, L, I, T(1), T(1), xi, true, false, sv, rp);
  }
}

// ------------------------------------------------------------------ the ADMM loop
// One iteration of Steps 1-4 (Sec. III-B) over the CTA's instance; all
// threads of the CTA call it.  The LAST instance also accumulates the primal
// and dual residuals (a separate instantiation, so that the hot loop carries
// no residual work, not even predicated off); their squared terms are summed
// in the wide type, per node and over the CTA (acc_sq_diff, reduce_residuals).
//
// GROUP: the CTA is one scenario of a group whose scenarios share the first
// control (Sec. IV-A).  After Step 3 the node-0 thread of every CTA publishes
// its Step-3 argument u_0 + nu_u,0 / rho_geo and its box (both absolute); the
// group all-reduce combines them, and each CTA sets u-hat_0 to the projection
// onto {equal u_0} intersected with every box, i.e. the average clamped to the
// common box, before its Step 4.
template <class M, class T, bool AOS, bool REFINE, bool LAST, bool GROUP, class MS, class NS>
__device__ __forceinline__ void admm_iteration(const Node<T, AOS>& nd, const MS& MT, const Layout& L, const Inst<T>& I,
                                               const NodeConst<M, T>& K, bool active, T re, T rd, T rg,
                                               T irg, T ired, typename WideOf<T>::type& rp,
                                               typename WideOf<T>::type& rdl, GroupShared* G,
                                               GroupX& X, const ProblemDev& P, const NS& S) {
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU;
  const int i = nd.i, N = nd.N;
  constexpr bool last = LAST;
  {
    T x[NN];
    // ---- Step 1: H_i xi_i = g_i with the cached factor (+ one refinement step).
    // Node N takes the same path: its factor carries an identity control block
    // with no coupling and its control rows of g are zero, so its control part
    // stays exactly zero and its state part is the state-only solve, while the
    // warp that holds it runs one code path instead of two.
    if (active) {
      T g[NN];
      node_rhs<M, T, AOS, NN>(nd, MT, L, I, K, S, re, rd, rg, g);
      sym_solve<T, NN>(MT, g, x);
      if constexpr (REFINE) {
        T hx[NN], dx[NN];
        apply_H<M, T, AOS, NN>(nd, MT, L, I, K, rd, rg, x, hx);
#pragma unroll
        for (int j = 0; j < NN; ++j) hx[j] = g[j] - hx[j];
        sym_solve<T, NN>(MT, hx, dx);
#pragma unroll
        for (int j = 0; j < NN; ++j) x[j] += dx[j];
      }
      if (i < N) {
        // linearised propagation d_dyn,i = A x + B u + c_i, published to node i+1
#pragma unroll
        for (int r = 0; r < NX; ++r) {
          T acc = nd.at(Rec<M>::C, r);
#pragma unroll
          for (int c = 0; c < NX; ++c) acc_A(acc, MT, r, c, x[c]);
#pragma unroll
          for (int c = 0; c < NU; ++c) acc += MT.B(r, c) * x[NX + c];
          nd.at(Rec<M>::Ex1, r) = acc;
        }
      }
#pragma unroll
      for (int j = 0; j < NX; ++j) nd.at(Rec<M>::X, j) = x[j];
      if (i < N) {
#pragma unroll
        for (int j = 0; j < NU; ++j) nd.at(Rec<M>::U, j) = x[NX + j];
      }
    }
    // Steps 2 and 3 use disjoint variables (z, lambda, mu | x-hat, u-hat, nu,
    // mirrors) and both read only this iteration's xi, so Step 3 runs first,
    // between the arrival on the split barrier (Ex1 published) and the wait
    // for the left neighbour's Ex1 that Step 2 needs: a warp that is ahead
    // projects instead of idling at a barrier.
    if constexpr (GROUP) __syncthreads();   // groups: their exchange follows Step 2 on a plain barrier
    else split_barrier_arrive(X.bar);
    T dz[NX];
    T sv[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) sv[j] = T(0);
    if (active) {
      // ---- Step 3: projections onto the boxes (Eq. (7)) and Step 4 for nu_x, nu_u
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        const T nux = S.nux(j);
        const T xh = clampv(x[j] + nux * irg, nd.at(Rec<M>::Xlo, j), nd.at(Rec<M>::Xhi, j));
        if (last) { sv[j] += rg * (xh - nd.at(Rec<M>::Xh, j)); acc_sq_diff(rp, x[j], xh); }
        nd.at(Rec<M>::Xh, j) = xh;
        S.nux(j) = nux + rg * (x[j] - xh);
      }
      if (i < N) {
#pragma unroll
        for (int j = 0; j < NU; ++j) {
          const T nuu = S.nuu(j);
          if constexpr (GROUP) {
            if (i == 0) {   // sum of arguments | max of lower bounds | max of -upper bounds
              const double ub = wide_to_double(nd.dat(Rec<M>::Ubar, j));
              double* m = G->mine[X.epoch & 1];
              m[j] = ub + (double)(x[NX + j] + nuu * irg);
              m[NU + j] = ub + (double)nd.at(Rec<M>::Ulo, j);
              m[2 * NU + j] = -(ub + (double)nd.at(Rec<M>::Uhi, j));
              continue;
            }
          }
          const T uh = clampv(x[NX + j] + nuu * irg, nd.at(Rec<M>::Ulo, j), nd.at(Rec<M>::Uhi, j));
          if (last) { sv[NX + j] += rg * (uh - nd.at(Rec<M>::Uh, j)); acc_sq_diff(rp, x[NX + j], uh); }
          nd.at(Rec<M>::Uh, j) = uh;
          S.nuu(j) = nuu + rg * (x[NX + j] - uh);
        }
      }
      node_mirrors<M, T, AOS, NN>(nd, L, I, rg, irg, x, false, last, sv, rp);   // control sets: i < N only
    }
    if constexpr (!GROUP) split_barrier_wait(X.bar, X.ph);
    if (active) {
      // ---- Step 2: dynamic consensus, Eq. (5), then its duals (Step 4)
      if (i >= 1) {
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          const T dd = nd.nb(Rec<M>::Ex1, j, i - 1);
          const T zo = S.z(j);
          const T lam = S.lam(j), mu = S.mu(j);
          const T z = (re * x[j] + lam + rd * dd - mu) * ired;
          S.z(j) = z;
          S.lam(j) = lam + re * (x[j] - z);
          const T mun = mu + rd * (z - dd);
          S.mu(j) = mun;
          dz[j] = z - zo;
          if (last) {
            sv[j] += re * dz[j];
            acc_sq_diff(rp, x[j], z); acc_sq_diff(rp, z, dd);
          }
        }
      }
    }
    if constexpr (GROUP) {
      double tot[3 * NU];
      group_allreduce<3 * NU>(P, G, X, NU, tot);
      if (active && i == 0 && i < N) {
#pragma unroll
        for (int j = 0; j < NU; ++j) {
          const double v = fmin(fmax(tot[j] / (double)P.group, tot[NU + j]), -tot[2 * NU + j]);
          G->u0[j] = v;
          const T uh = (T)(v - wide_to_double(nd.dat(Rec<M>::Ubar, j)));
          const T nuu = S.nuu(j);
          if (last) { sv[NX + j] += rg * (uh - nd.at(Rec<M>::Uh, j)); acc_sq_diff(rp, x[NX + j], uh); }
          nd.at(Rec<M>::Uh, j) = uh;
          S.nuu(j) = nuu + rg * (x[NX + j] - uh);
        }
      }
    }
    if constexpr (LAST) {
      // dual residual needs rho_dyn (z_{i+1,new} - z_{i+1,old}) from the right neighbour
      __syncthreads();
      if (active && i >= 1) {
#pragma unroll
        for (int j = 0; j < NX; ++j) nd.at(Rec<M>::Ex1, j) = rd * dz[j];
      }
      __syncthreads();
      if (active) {
        if (i < N) {
#pragma unroll
          for (int j = 0; j < NX; ++j) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < NX; ++k)
              if (MS::akind(k, j)) acc_A(acc, MT, k, j, nd.nb(Rec<M>::Ex1, k, i + 1));
            sv[j] += acc;
          }
#pragma unroll
          for (int j = 0; j < NU; ++j) {
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < NX; ++k) acc += MT.B(k, j) * nd.nb(Rec<M>::Ex1, k, i + 1);
            sv[NX + j] += acc;
          }
        }
#pragma unroll
        for (int j = 0; j < NN; ++j)
          if (j < NX || i < N) acc_sq(rdl, sv[j]);
      }
    }
    if (active && i >= 1) {
#pragma unroll
      for (int j = 0; j < NX; ++j) nd.at(Rec<M>::Ex2, j) = S.mu(j) + rd * S.z(j);
    }
    __syncthreads();
  }
}

// `iters` iterations of Steps 1-4; the primal and dual residuals of the last
// one are returned, squared, in res[0..1].
template <class M, class T, bool AOS, bool REFINE, bool GROUP = false, bool REGS = true, class MS>
__device__ __forceinline__ void admm_iterations(const Node<T, AOS>& nd, const MS& MT, const Layout& L, const Inst<T>& I,
                                const NodeConst<M, T>& K, bool active, T re, T rd, T rg, int iters,
                                InstShared& sh, double* res, GroupShared* G, GroupX& X, const ProblemDev& P) {
  const T irg = T(1) / rg, ired = T(1) / (re + rd);
  typename WideOf<T>::type rp{}, rdl{};   // residual sums in the wide type (FP64 or double-float)
  NodeStateFor<M, T, AOS, REGS> S;
  if (active) S.load(nd);
  for (int it = 0; it + 1 < iters; ++it)
    admm_iteration<M, T, AOS, REFINE, false, GROUP>(nd, MT, L, I, K, active, re, rd, rg, irg, ired, rp, rdl, G, X, P, S);
  admm_iteration<M, T, AOS, REFINE, true, GROUP>(nd, MT, L, I, K, active, re, rd, rg, irg, ired, rp, rdl, G, X, P, S);
  if (active) S.store(nd);
  // squared norms (the root is taken once, when they are reported)
  reduce_residuals(sh, rp, rdl, res);
}

// Publish mu_i + rho_dyn z_i before the first Step 1.
template <class M, class T, bool AOS>
__device__ __forceinline__ void publish_ex2(const Node<T, AOS>& nd, const Layout& L, bool active, T rd) {
  if (active && nd.i >= 1)
    for (int j = 0; j < M::NX; ++j) nd.at(Rec<M>::Ex2, j) = nd.at(Rec<M>::Mu, j) + rd * nd.at(Rec<M>::Z, j);
}

// Cold start: x = x-hat = z = nominal, u = u-hat = nominal, zero duals.
template <class M, class T, bool AOS>
__device__ void node_cold_start(const Node<T, AOS>& nd, const Layout& L) {
  for (int j = 0; j < M::NX; ++j) {
    nd.at(Rec<M>::X, j) = T(0); nd.at(Rec<M>::Z, j) = T(0); nd.at(Rec<M>::Lam, j) = T(0); nd.at(Rec<M>::Mu, j) = T(0);
    nd.at(Rec<M>::Xh, j) = T(0); nd.at(Rec<M>::Nux, j) = T(0);
  }
  for (int j = 0; j < M::NU; ++j) { nd.at(Rec<M>::U, j) = T(0); nd.at(Rec<M>::Uh, j) = T(0); nd.at(Rec<M>::Nuu, j) = T(0); }
  for (int j = 0; j < L.MS; ++j) { nd.at(L.oS, j) = T(0); nd.at(L.oNus, j) = T(0); }
}

// The ADMM state a solve starts from: cold (x = x-hat = z = nominal, zero
// duals), or -- warm[b] -- the absolute state in state_abs (a kept state of an
// earlier solve), taken relative to this solve's nominal.
template <class M, class T, bool AOS>
__device__ void node_import(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, int b, const double* in);
template <class M, class T, bool AOS>
__device__ __forceinline__ void node_start(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, int b) {
  if (P.warm && P.warm[b]) node_import<M, T, AOS>(nd, L, P, b, P.state_abs + P.soff[b]);
  else node_cold_start<M, T, AOS>(nd, L);
}

// ------------------------------------------------------------------ absolute state in/out
// Flat per-instance order: x, u, z, lam, mu, xh, uh, nux, nuu, s[(N+1)][MB][3], nus[...].
template <class M, class T, bool AOS>
__device__ void node_export(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, int b, double* out) {
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  const long long nX = (long long)(N + 1) * NX, nU = (long long)N * NU;
  double* px = out;           double* pu = px + nX;
  double* pz = pu + nU;       double* plam = pz + nX;
  double* pmu = plam + nX;    double* pxh = pmu + nX;
  double* puh = pxh + nX;     double* pnux = puh + nU;
  double* pnuu = pnux + nX;   double* ps = pnuu + nU;
  double* pnus = ps + (long long)(N + 1) * L.MB * 3;
  for (int j = 0; j < NX; ++j) {
    const double xb = wide_to_double(nd.dat(Rec<M>::Xbar, j));
    px[i * NX + j] = xb + (double)nd.at(Rec<M>::X, j);
    pz[i * NX + j] = (i >= 1) ? xb + (double)nd.at(Rec<M>::Z, j) : 0.0;
    plam[i * NX + j] = (i >= 1) ? (double)nd.at(Rec<M>::Lam, j) : 0.0;
    pmu[i * NX + j] = (i >= 1) ? (double)nd.at(Rec<M>::Mu, j) : 0.0;
    pxh[i * NX + j] = xb + (double)nd.at(Rec<M>::Xh, j);
    pnux[i * NX + j] = (double)nd.at(Rec<M>::Nux, j);
  }
  if (i < N)
    for (int j = 0; j < NU; ++j) {
      const double ub = wide_to_double(nd.dat(Rec<M>::Ubar, j));
      pu[i * NU + j] = ub + (double)nd.at(Rec<M>::U, j);
      puh[i * NU + j] = ub + (double)nd.at(Rec<M>::Uh, j);
      pnuu[i * NU + j] = (double)nd.at(Rec<M>::Nuu, j);
    }
  double* si = ps + (long long)i * L.MB * 3;
  double* ni = pnus + (long long)i * L.MB * 3;
  for (int k = 0; k < L.MB * 3; ++k) { si[k] = 0.0; ni[k] = 0.0; }
  if constexpr (IsQuad<M>::value) {
    for (int j = 0; j < nobs_of(P, b); ++j) {
      double np = 0.0;
      for (int k = 0; k < 3; ++k) np += (double)nd.at(L.oMd, ObsStride<T>::value * j + k) * wide_to_double(nd.dat(Rec<M>::Xbar, k));
      si[3 * j] = (double)nd.at(L.oS, j) + np;
      ni[3 * j] = (double)nd.at(L.oNus, j);
    }
  } else if constexpr (IsMars14<M>::value) {
    // blocks as the problem's sets: glide cone, tilt, body rate, thrust ball, thrust lower bound, gimbal
    const double* st = &P.sets[b * UCN_SET_PARAMS];
    if (st[2] > 0.0)
      for (int k = 0; k < 3; ++k) { si[k] = (double)nd.at(L.oS, k) + wide_to_double(nd.dat(Rec<M>::Xbar, 1 + k)); ni[k] = (double)nd.at(L.oNus, k); }
    if (st[4] > 0.0)
      for (int k = 0; k < 2; ++k) {
        si[3 + k] = (double)nd.at(L.oS, M14::S_TILT + k) + wide_to_double(nd.dat(Rec<M>::Xbar, 9 + k));
        ni[3 + k] = (double)nd.at(L.oNus, M14::S_TILT + k);
      }
    if (st[5] > 0.0)
      for (int k = 0; k < 3; ++k) {
        si[6 + k] = (double)nd.at(L.oS, M14::S_W + k) + wide_to_double(nd.dat(Rec<M>::Xbar, 11 + k));
        ni[6 + k] = (double)nd.at(L.oNus, M14::S_W + k);
      }
    if (i < N && st[1] > 0.0)
      for (int k = 0; k < 3; ++k) { si[9 + k] = (double)nd.at(L.oS, 3 + k) + wide_to_double(nd.dat(Rec<M>::Ubar, k)); ni[9 + k] = (double)nd.at(L.oNus, 3 + k); }
    if (i < N && st[0] > 0.0) {
      double np = 0.0;
      for (int k = 0; k < 3; ++k) np += (double)nd.at(L.oMd, k) * wide_to_double(nd.dat(Rec<M>::Ubar, k));
      si[12] = (double)nd.at(L.oS, 6) + np;
      ni[12] = (double)nd.at(L.oNus, 6);
    }
    if (i < N && st[3] > 0.0)
      for (int k = 0; k < 3; ++k) {
        si[15 + k] = (double)nd.at(L.oS, M14::S_GIM + k) + wide_to_double(nd.dat(Rec<M>::Ubar, k));
        ni[15 + k] = (double)nd.at(L.oNus, M14::S_GIM + k);
      }
  } else {
    if (P.sets[b * UCN_SET_PARAMS + 2] > 0.0)
      for (int k = 0; k < 3; ++k) { si[k] = (double)nd.at(L.oS, k) + wide_to_double(nd.dat(Rec<M>::Xbar, k)); ni[k] = (double)nd.at(L.oNus, k); }
    if (i < N && P.sets[b * UCN_SET_PARAMS + 1] > 0.0)
      for (int k = 0; k < 3; ++k) { si[3 + k] = (double)nd.at(L.oS, 3 + k) + wide_to_double(nd.dat(Rec<M>::Ubar, k)); ni[3 + k] = (double)nd.at(L.oNus, 3 + k); }
    if (i < N && P.sets[b * UCN_SET_PARAMS + 0] > 0.0) {
      double np = 0.0;
      for (int k = 0; k < 3; ++k) np += (double)nd.at(L.oMd, k) * wide_to_double(nd.dat(Rec<M>::Ubar, k));
      si[6] = (double)nd.at(L.oS, 6) + np;
      ni[6] = (double)nd.at(L.oNus, 6);
    }
  }
}

template <class M, class T, bool AOS>
__device__ void node_import(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, int b, const double* in) {
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  const long long nX = (long long)(N + 1) * NX, nU = (long long)N * NU;
  const double* px = in;          const double* pu = px + nX;
  const double* pz = pu + nU;     const double* plam = pz + nX;
  const double* pmu = plam + nX;  const double* pxh = pmu + nX;
  const double* puh = pxh + nX;   const double* pnux = puh + nU;
  const double* pnuu = pnux + nX; const double* ps = pnuu + nU;
  const double* pnus = ps + (long long)(N + 1) * L.MB * 3;
  for (int j = 0; j < NX; ++j) {
    const double xb = wide_to_double(nd.dat(Rec<M>::Xbar, j));
    nd.at(Rec<M>::X, j) = (T)(px[i * NX + j] - xb);
    nd.at(Rec<M>::Z, j) = (i >= 1) ? (T)(pz[i * NX + j] - xb) : T(0);
    nd.at(Rec<M>::Lam, j) = (T)plam[i * NX + j];
    nd.at(Rec<M>::Mu, j) = (T)pmu[i * NX + j];
    nd.at(Rec<M>::Xh, j) = (T)(pxh[i * NX + j] - xb);
    nd.at(Rec<M>::Nux, j) = (T)pnux[i * NX + j];
  }
  for (int j = 0; j < NU; ++j) {
    const double ub = (i < N) ? wide_to_double(nd.dat(Rec<M>::Ubar, j)) : 0.0;
    nd.at(Rec<M>::U, j) = (i < N) ? (T)(pu[i * NU + j] - ub) : T(0);
    nd.at(Rec<M>::Uh, j) = (i < N) ? (T)(puh[i * NU + j] - ub) : T(0);
    nd.at(Rec<M>::Nuu, j) = (i < N) ? (T)pnuu[i * NU + j] : T(0);
  }
  for (int j = 0; j < L.MS; ++j) { nd.at(L.oS, j) = T(0); nd.at(L.oNus, j) = T(0); }
  const double* si = ps + (long long)i * L.MB * 3;
  const double* ni = pnus + (long long)i * L.MB * 3;
  if constexpr (IsQuad<M>::value) {
    for (int j = 0; j < nobs_of(P, b); ++j) {
      double np = 0.0;
      for (int k = 0; k < 3; ++k) np += (double)nd.at(L.oMd, ObsStride<T>::value * j + k) * wide_to_double(nd.dat(Rec<M>::Xbar, k));
      nd.at(L.oS, j) = (T)(si[3 * j] - np);
      nd.at(L.oNus, j) = (T)ni[3 * j];
    }
  } else if constexpr (IsMars14<M>::value) {
    // blocks as exported: glide cone, tilt, body rate, thrust ball, thrust lower bound, gimbal
    for (int k = 0; k < 3; ++k) { nd.at(L.oS, k) = (T)(si[k] - wide_to_double(nd.dat(Rec<M>::Xbar, 1 + k))); nd.at(L.oNus, k) = (T)ni[k]; }
    for (int k = 0; k < 2; ++k) {
      nd.at(L.oS, M14::S_TILT + k) = (T)(si[3 + k] - wide_to_double(nd.dat(Rec<M>::Xbar, 9 + k)));
      nd.at(L.oNus, M14::S_TILT + k) = (T)ni[3 + k];
    }
    for (int k = 0; k < 3; ++k) {
      nd.at(L.oS, M14::S_W + k) = (T)(si[6 + k] - wide_to_double(nd.dat(Rec<M>::Xbar, 11 + k)));
      nd.at(L.oNus, M14::S_W + k) = (T)ni[6 + k];
    }
    if (i < N) {
      for (int k = 0; k < 3; ++k) { nd.at(L.oS, 3 + k) = (T)(si[9 + k] - wide_to_double(nd.dat(Rec<M>::Ubar, k))); nd.at(L.oNus, 3 + k) = (T)ni[9 + k]; }
      double np = 0.0;
      for (int k = 0; k < 3; ++k) np += (double)nd.at(L.oMd, k) * wide_to_double(nd.dat(Rec<M>::Ubar, k));
      nd.at(L.oS, 6) = (T)(si[12] - np);
      nd.at(L.oNus, 6) = (T)ni[12];
      for (int k = 0; k < 3; ++k) {
        nd.at(L.oS, M14::S_GIM + k) = (T)(si[15 + k] - wide_to_double(nd.dat(Rec<M>::Ubar, k)));
        nd.at(L.oNus, M14::S_GIM + k) = (T)ni[15 + k];
      }
    }
  } else {
    for (int k = 0; k < 3; ++k) { nd.at(L.oS, k) = (T)(si[k] - wide_to_double(nd.dat(Rec<M>::Xbar, k))); nd.at(L.oNus, k) = (T)ni[k]; }
    if (i < N) {
      for (int k = 0; k < 3; ++k) { nd.at(L.oS, 3 + k) = (T)(si[3 + k] - wide_to_double(nd.dat(Rec<M>::Ubar, k))); nd.at(L.oNus, 3 + k) = (T)ni[3 + k]; }
      double np = 0.0;
      for (int k = 0; k < 3; ++k) np += (double)nd.at(L.oMd, k) * wide_to_double(nd.dat(Rec<M>::Ubar, k));
      nd.at(L.oS, 6) = (T)(si[6] - np);
      nd.at(L.oNus, 6) = (T)ni[6];
    }
  }
}

// After an accepted step the nominal moves by (dxh, duh): express the mirror
// variables in deviations from the new nominal (same absolute values).
template <class M, class T, bool AOS>
__device__ void node_rebase_mirrors(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, int b) {
  if constexpr (IsQuad<M>::value) {
    for (int j = 0; j < nobs_of(P, b); ++j) {
      T y = T(0);
      for (int k = 0; k < 3; ++k) y += nd.at(L.oMd, ObsStride<T>::value * j + k) * nd.at(Rec<M>::Xh, k);
      nd.at(L.oS, j) -= y;
    }
  } else {
    constexpr int RC = IsMars14<M>::value ? 1 : 0;
    for (int k = 0; k < 3; ++k) nd.at(L.oS, k) -= nd.at(Rec<M>::Xh, RC + k);
    if constexpr (IsMars14<M>::value) {
      for (int k = 0; k < 2; ++k) nd.at(L.oS, M14::S_TILT + k) -= nd.at(Rec<M>::Xh, 9 + k);
      for (int k = 0; k < 3; ++k) nd.at(L.oS, M14::S_W + k) -= nd.at(Rec<M>::Xh, 11 + k);
    }
    if (nd.i < nd.N) {
      T y = T(0);
      for (int k = 0; k < 3; ++k) { nd.at(L.oS, 3 + k) -= nd.at(Rec<M>::Uh, k); y += nd.at(L.oMd, k) * nd.at(Rec<M>::Uh, k); }
      nd.at(L.oS, 6) -= y;
      if constexpr (IsMars14<M>::value)
        for (int k = 0; k < 3; ++k) nd.at(L.oS, M14::S_GIM + k) -= nd.at(Rec<M>::Uh, k);
    }
  }
}

// ------------------------------------------------------------------ kernels
template <class T, bool SMEM>
__device__ __forceinline__ Node<T, SMEM> make_node(const ProblemDev& P, const Layout& L, unsigned char* smem, int b) {
  unsigned char* base = SMEM ? smem : (unsigned char*)(P.ws + (long long)b * L.bytes);
  Node<T, SMEM> nd;
  nd.t = (T*)base;
  nd.d = (typename Node<T, SMEM>::W*)(base + L.tbytes);
  nd.c = L.oC >= 0 ? (typename Node<T, SMEM>::W*)(base + L.oC) : nullptr;
  nd.S = L.S;
  nd.NS = L.NS;
  nd.DS = L.DS;
  nd.i = threadIdx.x;
  nd.N = P.N[b];
  return nd;
}

// Linearisation of every node of every instance (one thread per control node).
template <class M, class T>
__global__ void __launch_bounds__(128) linearize_kernel(ProblemDev P, const int* node_inst, long long total_u,
                                                        const double* xbar, const double* ubar,
                                                        double* A, double* B, double* d) {
  constexpr int NX = M::NX, NU = M::NU;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total_u) return;
  const int b = node_inst[g];
  const long long i = g - P.uoff[b];
  const long long xr = P.xoff[b] + i;
  double x[NX], u[NU];
  for (int j = 0; j < NX; ++j) x[j] = xbar[xr * NX + j];
  for (int j = 0; j < NU; ++j) u[j] = ubar[g * NU + j];
  const double* prm = P.params + b * 8;
  const double h = P.dt[b];
  double Ad[NX * NX], Bd[NX * NU];
  for (int dir = 0; dir < NX + NU; ++dir) {
    T col[NX];
    rk4_jvp<M, T>(prm, step_of<T>(h), x, u, dir, col);
    for (int r = 0; r < NX; ++r) {
      if (dir < NX) Ad[r * NX + dir] = (double)col[r];
      else Bd[r * NU + dir - NX] = (double)col[r];
    }
  }
  double xn[NX];
  rk4<M, double>(prm, h, x, u, xn);
  for (int r = 0; r < NX; ++r) {
    double acc = xn[r];
    for (int c = 0; c < NX; ++c) acc -= Ad[r * NX + c] * x[c];
    for (int c = 0; c < NU; ++c) acc -= Bd[r * NU + c] * u[c];
    d[g * NX + r] = acc;
  }
  for (int e = 0; e < NX * NX; ++e) A[g * NX * NX + e] = Ad[e];
  for (int e = 0; e < NX * NU; ++e) B[g * NX * NU + e] = Bd[e];
}

// Standalone ADMM call on caller-supplied linearisations (one CTA per instance).
template <class M, class T, bool SMEM, bool REFINE>
__global__ void __launch_bounds__(MAX_THREADS) admm_kernel(ProblemDev P, Layout L, const double* xbar, const double* ubar,
                                                           const double* Ag, const double* Bg, const double* dg,
                                                           const double* radius, int iters, int warm,
                                                           double* xhat, double* uhat, double* res, int* status) {
  constexpr int NX = M::NX, NU = M::NU;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ InstShared sh;
  const int b = blockIdx.x;
  constexpr bool AOS = SMEM;
  Node<T, AOS> nd = make_node<T, SMEM>(P, L, smem, b);
  MatsFor<M, T, AOS> MT;
  init_mats<M, T, AOS>(MT, nd, L);
  const int i = nd.i, N = nd.N;
  const bool active = i <= N;
  const long long xo = P.xoff[b], uo = P.uoff[b];
  if (threadIdx.x == 0) { sh.fail = 0; split_barrier_init(sh.xbar, blockDim.x); }
  stage_consts<M, T, AOS>(nd, P, b);
  if (active) load_nominal<M, T, AOS>(nd, L, xbar, ubar, xo, uo);
  __syncthreads();
  if (active && i < N) {
    // A, B in T; deviation affine term c_i = A xbar_i + B ubar_i + d_i - xbar_{i+1} in FP64 (once per call)
    const long long g = uo + i;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
#pragma unroll
      for (int c = 0; c < NX; ++c) MT.A(r, c) = (T)Ag[g * NX * NX + r * NX + c];
#pragma unroll
      for (int c = 0; c < NU; ++c) MT.B(r, c) = (T)Bg[g * NX * NU + r * NU + c];
    }
    for (int r = 0; r < NX; ++r) {
      double acc = dg[g * NX + r];
      for (int c = 0; c < NX; ++c) acc += Ag[g * NX * NX + r * NX + c] * wide_to_double(nd.dat(Rec<M>::Xbar, c));
      for (int c = 0; c < NU; ++c) acc += Bg[g * NX * NU + r * NU + c] * wide_to_double(nd.dat(Rec<M>::Ubar, c));
      nd.at(Rec<M>::C, r) = (T)(acc - wide_to_double(nd.dnb(Rec<M>::Xbar, r, i + 1)));
    }
  }
  const T re = (T)P.rho_eq, rd = (T)P.rho_dyn, rg = (T)P.rho_geo;
  const Inst<T> I = make_inst<M, T>(P, b);
  NodeConst<M, T> K;
  if (active) {
    node_setup<M, T, AOS>(nd, L, P, I, b, radius[b], re, rg, K);
    const bool ok = node_factor<M, T, AOS, NX + NU>(nd, MT, L, I, K, rd, rg);
    if (!ok) atomicOr(&sh.fail, 1);
    const double* sa = P.state_abs + P.soff[b];
    if (warm) {
      node_import<M, T, AOS>(nd, L, P, b, sa);
    } else {
      node_cold_start<M, T, AOS>(nd, L);
      node_reseed<M, T, AOS>(nd, L, I);
    }
    publish_ex2<M, T, AOS>(nd, L, active, rd);
  }
  __syncthreads();
  double r2[2] = {0.0, 0.0};
  GroupX X{0u, 0, 0, sh.xbar, 0u};
  if (!sh.fail) admm_iterations<M, T, AOS, REFINE>(nd, MT, L, I, K, active, re, rd, rg, iters, sh, r2, nullptr, X, P);
  if (active) {
    node_export<M, T, AOS>(nd, L, P, b, P.state_abs + P.soff[b]);
    for (int j = 0; j < NX; ++j) xhat[(xo + i) * NX + j] = wide_to_double(nd.dat(Rec<M>::Xbar, j)) + (double)nd.at(Rec<M>::Xh, j);
    if (i < N)
      for (int j = 0; j < NU; ++j) uhat[(uo + i) * NU + j] = wide_to_double(nd.dat(Rec<M>::Ubar, j)) + (double)nd.at(Rec<M>::Uh, j);
  }
  if (threadIdx.x == 0) {
    res[2 * b] = sqrt(r2[0]);
    res[2 * b + 1] = sqrt(r2[1]);
    status[b] = (sh.fail || sh.xbar[1]) ? ST_NUMERIC : ST_OK;
  }
}

// Nonlinear cost l(x_i,u_i) (or phi(x_N)) of node i in the wide type (FP64
// from the problem arrays, or double-float from the CB block).
template <class M, class T, bool AOS>
__device__ __forceinline__ typename Node<T, AOS>::W node_cost(const Node<T, AOS>& nd, const ProblemDev& P,
                                                              const Inst<T>& I, int b, int i, int N,
                                                              const typename Node<T, AOS>::W* x,
                                                              const typename Node<T, AOS>::W* u) {
  constexpr int NX = M::NX, NU = M::NU;
  if constexpr (IsDF<T>::value) {
    typedef CB<M> C;
    const DF* cb = nd.c;
    DF c;
    if (i == N && !I.term_quad) {
      for (int j = 0; j < NX; ++j) c = df_add(c, df_mul(cb[C::QN + j], x[j]));
      return c;
    }
    if (i < N && !I.run_cost) return c;
    if (i < N) {
      for (int j = 0; j < NX; ++j) {
        const DF e = df_sub(x[j], cb[C::Xref + j]);
        c = df_add(c, df_mul(df_mul(e, e), df_mul(cb[C::Qd + j], 0.5f)));
      }
      for (int j = 0; j < NU; ++j) {
        const DF e = df_sub(u[j], cb[C::Uref + j]);
        c = df_add(c, df_mul(df_mul(e, e), df_mul(cb[C::Rd + j], 0.5f)));
      }
    } else {
      for (int j = 0; j < NX; ++j) {
        const DF e = df_sub(x[j], cb[C::Xref + j]);
        c = df_add(c, df_add(df_mul(df_mul(e, e), df_mul(cb[C::QNd + j], 0.5f)), df_mul(cb[C::QN + j], x[j])));
      }
    }
    return c;
  } else {
  double c = 0.0;
  if (i == N && !I.term_quad) {
    for (int j = 0; j < NX; ++j) c += P.qN[b * NX + j] * x[j];
    return c;
  }
  if (i < N && !I.run_cost) return 0.0;
  if (i < N) {
    for (int j = 0; j < NX; ++j) { const double e = x[j] - P.xref[b * NX + j]; c += 0.5 * P.Qd[b * NX + j] * e * e; }
    for (int j = 0; j < NU; ++j) { const double e = u[j] - P.uref[b * NU + j]; c += 0.5 * P.Rd[b * NU + j] * e * e; }
  } else {
    for (int j = 0; j < NX; ++j) {
      const double e = x[j] - P.xref[b * NX + j];
      c += 0.5 * P.QNd[b * NX + j] * e * e + P.qN[b * NX + j] * x[j];
    }
  }
  return c;
  }
}

// ------------------------------------------------------------------ per-SCP-iteration steps
// The steps of an SCP iteration outside the ADMM loop, shared by the fused
// kernels (one thread per node, `act` when the thread has one; every thread of
// the CTA calls them).  Wide arithmetic: FP64, or double-float on the FP32
// path, whose sums are reduced in double-float and handed over as doubles.

// Input check of one instance, by all threads of its CTA (after sh.fail is
// cleared, before the first factorisation): a NaN anywhere in its data or
// guesses, or an infinity where only finite values have a meaning (everything
// but the state and control bounds and the set parameters, where +-inf means
// "no bound"), sets sh.fail, so the solve stops after its first factorisation
// with UCN_ENUMERIC instead of iterating on garbage.  Other instances of the
// launch are not touched.
template <class M>
__device__ void flag_bad_inputs(const ProblemDev& P, int b, const double* x0, const double* u0, long long xo,
                                long long uo, InstShared& sh) {
  const int nx = P.nx, nu = P.nu, N = P.N[b];
  const int no = IsQuad<M>::value ? nobs_of(P, b) : 0;
  struct Span { const double* p; int n; bool finite; };
  const Span sp[] = {
      {P.dt + b, 1, true}, {P.params + 8 * b, 8, true}, {P.Qd + b * nx, nx, true}, {P.xref + b * nx, nx, true},
      {P.Rd + b * nu, nu, true}, {P.uref + b * nu, nu, true}, {P.QNd + b * nx, nx, true}, {P.qN + b * nx, nx, true},
      {P.xinit + b * nx, nx, true}, {P.xtarget + b * nx, nx, true}, {P.xlo + b * nx, nx, false},
      {P.xhi + b * nx, nx, false}, {P.ulo + b * nu, nu, false}, {P.uhi + b * nu, nu, false},
      {P.sets + b * UCN_SET_PARAMS, UCN_SET_PARAMS, false}, {x0 + xo * nx, (N + 1) * nx, true},
      {u0 + uo * nu, N * nu, true}, {P.obs_c + (long long)b * P.max_obs * 3, 3 * no, true},
      {P.obs_r + (long long)b * P.max_obs, no, true}};
  bool bad = false;
  for (const Span& q : sp)
    for (int e = threadIdx.x; e < q.n; e += blockDim.x) {
      const double v = q.p[e];
      bad |= q.finite ? !isfinite(v) : isnan(v);
    }
  if (bad) atomicOr(&sh.fail, 1);
}

// Start of a solve: c_i = RK4(xbar_i, ubar_i) - xbar_{i+1} and J(nominal) in sh.Jn.
template <class M, class T, bool AOS>
__device__ void scp_start(const Node<T, AOS>& nd, const ProblemDev& P, const Inst<T>& I, int b, bool act,
                          InstShared& sh) {
  typedef typename Node<T, AOS>::W W;
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  W ac[2] = {W(), W()};
  if (act) {
    W xb[NX], ub[NU];
    read_nominal<M, T, AOS>(nd, i < N, xb, ub);
    ac[0] = node_cost<M, T, AOS>(nd, P, I, b, i, N, xb, ub);
    if (i < N) {
      W fn[NX];
      rk4_wide<M, T, AOS>(nd, P, b, xb, ub, fn);
      for (int j = 0; j < NX; ++j) {
        const W e = fn[j] - nd.dnb(Rec<M>::Xbar, j, i + 1);
        nd.at(Rec<M>::C, j) = wide_to<T>(e);
        ac[1] = ac[1] + wide_abs(e);
      }
    }
  }
  if constexpr (IsDF<T>::value) {
    block_reduce_df(sh, ac, 2, nullptr, 0, acc);
  } else {
    acc[0] = ac[0]; acc[1] = ac[1];
    block_reduce(sh, acc, 2, 2);
  }
  if (threadIdx.x == 0) sh.Jn = acc[0] + P.w_d * acc[1];
}

// The candidate (x-hat, u-hat) of an SCP iteration: its trajectory (xc, uc),
// defects fc_i = RK4(xc_i, uc_i) - xc_{i+1}, and CTA totals in v: cost, l1
// defect, l1 defect of the linear model | max defect, max step.
template <class M, class T, bool AOS, bool GROUP, class MS>
__device__ void scp_candidate(const Node<T, AOS>& nd, const MS& MT, const ProblemDev& P, const Inst<T>& I, int b,
                              bool act, const GroupShared* G, InstShared& sh, typename Node<T, AOS>::W* xc,
                              typename Node<T, AOS>::W* uc, typename Node<T, AOS>::W* fc, double* v) {
  typedef typename Node<T, AOS>::W W;
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  if (act) {
    for (int j = 0; j < NX; ++j) { xc[j] = wide_add(nd.dat(Rec<M>::Xbar, j), nd.at(Rec<M>::Xh, j)); nd.dat(Rec<M>::Xc, j) = xc[j]; }
    for (int j = 0; j < NU; ++j) uc[j] = (i < N) ? wide_add(nd.dat(Rec<M>::Ubar, j), nd.at(Rec<M>::Uh, j)) : W();
    if constexpr (GROUP) {
      // the shared first control exactly (bitwise equal across the group)
      if (i == 0)
        for (int j = 0; j < NU; ++j) uc[j] = wide_from_double<W>(G->u0[j]);
    }
  }
  __syncthreads();
  W vs[3] = {W(), W(), W()};                    // cost, nl1, lin1
  decltype(wide_abs_round(W())) dinf = 0;       // max |defect|
  T st = T(0), lin1 = T(0);
  if (act) {
    vs[0] = node_cost<M, T, AOS>(nd, P, I, b, i, N, xc, uc);
    for (int j = 0; j < NX; ++j) st = maxv(st, absv(nd.at(Rec<M>::Xh, j)));
    if (i < N) {
      for (int j = 0; j < NU; ++j) st = maxv(st, absv(nd.at(Rec<M>::Uh, j)));
      rk4_wide<M, T, AOS>(nd, P, b, xc, uc, fc);
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        fc[r] = fc[r] - nd.dnb(Rec<M>::Xc, r, i + 1);
        vs[1] = vs[1] + wide_abs(fc[r]);
        dinf = maxv(dinf, wide_abs_round(fc[r]));
        T lin = nd.at(Rec<M>::C, r) - nd.nb(Rec<M>::Xh, r, i + 1);
#pragma unroll
        for (int c = 0; c < NX; ++c)
          if (MS::akind(r, c)) acc_A(lin, MT, r, c, nd.at(Rec<M>::Xh, c));
#pragma unroll
        for (int c = 0; c < NU; ++c) lin += MT.B(r, c) * nd.at(Rec<M>::Uh, c);
        lin1 += absv(lin);
      }
    }
  }
  if constexpr (IsDF<T>::value) {
    vs[2] = df_from(lin1);
    float mx[2] = {dinf, st};
    block_reduce_df(sh, vs, 3, mx, 2, v);
  } else {
    v[0] = vs[0]; v[1] = vs[1]; v[2] = (double)lin1; v[3] = dinf; v[4] = (double)st;
    block_reduce(sh, v, 3, 5);
  }
}

// Accepted: the candidate becomes the nominal, its defect becomes c_i, and the
// deviations are re-based on it.
template <class M, class T, bool AOS>
__device__ void scp_move_nominal(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, int b,
                                 const typename Node<T, AOS>::W* xc, const typename Node<T, AOS>::W* uc,
                                 const typename Node<T, AOS>::W* fc) {
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  node_rebase_mirrors<M, T, AOS>(nd, L, P, b);
  for (int j = 0; j < NX; ++j) {
    const T xh = nd.at(Rec<M>::Xh, j);
    nd.dat(Rec<M>::Xbar, j) = xc[j];
    nd.at(Rec<M>::X, j) -= xh;
    if (i >= 1) nd.at(Rec<M>::Z, j) -= xh;
    nd.at(Rec<M>::Xh, j) = T(0);
    if (i < N) nd.at(Rec<M>::C, j) = wide_to<T>(fc[j]);
  }
  if (i < N)
    for (int j = 0; j < NU; ++j) {
      const T uh = nd.at(Rec<M>::Uh, j);
      nd.dat(Rec<M>::Ubar, j) = uc[j];
      nd.at(Rec<M>::U, j) -= uh;
      nd.at(Rec<M>::Uh, j) = T(0);
    }
}

// End of a solve: the returned (last accepted) trajectory, its cost, l1 and
// max defect (w[0..2], CTA totals; the defects by FP64 RK4 steps and FP64
// sums: once per launch) and the exported ADMM state.
template <class M, class T, bool AOS>
__device__ void scp_finish(const Node<T, AOS>& nd, const Layout& L, const ProblemDev& P, const Inst<T>& I, int b,
                           bool act, long long xo, long long uo, double* xout, double* uout, InstShared& sh,
                           double* w) {
  typedef typename Node<T, AOS>::W W;
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  if (act) {
    W xb[NX], ub[NU];
    read_nominal<M, T, AOS>(nd, i < N, xb, ub);
    w[0] = wide_to_double(node_cost<M, T, AOS>(nd, P, I, b, i, N, xb, ub));
    // the returned trajectory as doubles
    double xd[NX], ud[NU];
    for (int j = 0; j < NX; ++j) {
      xd[j] = wide_to_double(xb[j]);
      // a node-0 state at the initial state (Eq. (1c)) is returned bit for bit
      // as given, although double-float holds only ~48 of its 53 bits
      if constexpr (IsDF<T>::value)
        if (i == 0 && df_sub(nd.c[CB<M>::Xinit + j], xb[j]).hi == 0.0f) xd[j] = P.xinit[b * NX + j];
      xout[(xo + i) * NX + j] = xd[j];
    }
    for (int j = 0; j < NU; ++j) ud[j] = (i < N) ? wide_to_double(ub[j]) : 0.0;
    if (i < N) {
      for (int j = 0; j < NU; ++j) uout[(uo + i) * NU + j] = ud[j];
      // the defect of the returned trajectory by an FP64 RK4 step on both paths
      // (once per launch): the reported defect and the defect_tol status are
      // FP64 quantities of exactly the doubles returned
      double fn[NX];
      rk4<M, double>(P.params + b * 8, P.dt[b], xd, ud, fn);
      for (int j = 0; j < NX; ++j) {
        const double e = fabs(fn[j] - wide_to_double(nd.dnb(Rec<M>::Xbar, j, i + 1)));
        w[1] += e;
        w[2] = fmax(w[2], e);
      }
    }
    node_export<M, T, AOS>(nd, L, P, b, P.state_abs + P.soff[b]);
  }
  block_reduce(sh, w, 2, 3);
}

// The acceptance test and trust-region update of one SCP iteration (the paper
// omits them, Sec. III-A; ratio test on an l1 merit), by one thread: J(nominal)
// Jn, J(candidate) Jc, the linear model L(candidate) Lc (sums over a scenario
// group where there is one, Jc_own this CTA's own J(candidate)), the
// candidate's max defect and step; sets sh.accept, sh.radius, sh.Jn, sh.stop
// and sh.status.
__device__ __forceinline__ void scp_decide(InstShared& sh, const ProblemDev& P, double Jn, double Jc, double Lc,
                                           double Jc_own, double dinf, double step, bool timed_out, int k, int Kscp) {
  const double den = Jn - Lc, num = Jn - Jc;
  double radius2 = sh.radius;
  bool acc_ = true;
  if (!(den <= 1e-12)) {
    const double ratio = num / den;
    acc_ = ratio > 0.0;
    if (ratio < 0.25) radius2 *= 0.5;
    else if (ratio > 0.75) radius2 = fmin(2.0 * radius2, P.tr_max);
  }
  radius2 = fmax(radius2, P.tr_min);
  if (!isfinite(Jc)) { acc_ = false; sh.status = ST_NUMERIC; }
  if (acc_) sh.Jn = Jc_own;
  sh.radius = radius2;
  sh.accept = acc_;
  int stop = (sh.status == ST_NUMERIC);
  if (P.stop && acc_ && dinf <= P.defect_tol && step <= P.step_tol) stop = 1;
  if (timed_out && !stop && k + 1 < Kscp) { sh.status = ST_TIMEOUT; stop = 1; }
  sh.stop = stop;
}

// The per-instance result record and status of a solve, by one thread; w: the
// returned trajectory's cost, l1 and max defect (scp_finish); group_failed: a
// scenario group lost its consensus partner.
__device__ __forceinline__ void scp_report(const InstShared& sh, const ProblemDev& P, int b, const double* w,
                                           const double* res, double last_step, int iters_run, int accepted,
                                           unsigned long long mask, unsigned long long t0, bool group_failed,
                                           ucn_scp_stats* stats, int* status_out) {
  int st = sh.status;
  if (group_failed && st != ST_NUMERIC) st = ST_TIMEOUT;
  if (!isfinite(w[2]) || sh.xbar[1]) st = ST_NUMERIC;
  if (st == ST_OK && !(w[2] <= P.defect_tol)) st = ST_NOTCONV;
  ucn_scp_stats s;
  s.defect = w[2]; s.cost = w[0]; s.merit = w[0] + P.w_d * w[1];
  s.primal_res = sqrt(res[0]); s.dual_res = sqrt(res[1]); s.tr_radius = sh.radius; s.step = last_step;
  s.scp_iters = iters_run; s.accepted = accepted; s.accept_mask = mask; s.status = st; s.reserved = 0;
  s.t_start_ns = t0; s.t_end_ns = globaltimer_ns();
  s.pad[0] = s.pad[1] = s.pad[2] = s.pad[3] = 0.0;
  stats[b] = s;
  status_out[b] = st;
}

// The whole SCP solve of one instance per CTA (Sec. III-A + III-B): per SCP
// iteration, linearise (T), assemble + factor (T), admm_iters ADMM
// iterations (T), then the rollout, defects, merit and trust-region
// acceptance and the nominal update in the wide type (FP64, or double-float on
// the FP32 path) -- without leaving the kernel.
//
// GROUP: CTA k of group g solves scenario k of problem g (instance g * group
// + k); the group's CTAs are launched as thread-block clusters so that they are
// resident together.  The scenarios run their ADMM iterations in lockstep with
// the first-control consensus and take every decision as a group: a
// factorisation failure anywhere stops the group, and acceptance, trust
// radius, stopping and the time budget are decided on the group's sums
// (merits) and maxima (defect, step), so that accepted nominals keep one first
// control.
//
// REGS = false: the ADMM state stays in the node records (the variant that runs
// three CTAs per SM has no registers for it).
template <class M, class T, bool SMEM, bool REFINE, bool GROUP, bool REGS>
__device__ __forceinline__ void scp_body(const ProblemDev& P, const Layout& L, const double* x0, const double* u0,
                                         double* xout, double* uout, ucn_scp_stats* stats, int* status_out,
                                         const int b) {
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU;
  static_assert(!GROUP || NU <= 4, "GroupShared holds nu <= 4");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ InstShared sh;
  GroupShared* G = group_slot<GROUP>();
  GroupX X{0u, 0, 0};
  if constexpr (GROUP) {
    X.g = (int)blockIdx.x / P.group;
    X.k = (int)blockIdx.x % P.group;
    if (threadIdx.x == 0) G->gfail = 0;
  }
  constexpr bool AOS = SMEM;
  Node<T, AOS> nd = make_node<T, SMEM>(P, L, smem, b);
  MatsFor<M, T, AOS, true> MT;
  init_mats<M, T, AOS>(MT, nd, L);
  typedef typename Node<T, AOS>::W W;
  const int i = nd.i, N = nd.N;
  const bool active = i <= N;
  const long long xo = P.xoff[b], uo = P.uoff[b];
  const Step3<T> hs = step_of<T>(P.dt[b]);   // the RK4 step in T, once per launch
  const unsigned long long t0 = globaltimer_ns();
  const Inst<T> I = make_inst<M, T>(P, b);
  NodeConst<M, T> K;
  if (threadIdx.x == 0) {
    sh.fail = 0; sh.status = ST_OK; sh.radius = P.tr_init; sh.stop = 0;
    split_barrier_init(sh.xbar, blockDim.x);
  }
  X.bar = sh.xbar;
  stage_consts<M, T, AOS>(nd, P, b);
  if (active) load_nominal<M, T, AOS>(nd, L, x0, u0, xo, uo);
  __syncthreads();
  flag_bad_inputs<M>(P, b, x0, u0, xo, uo, sh);
  scp_start<M, T, AOS>(nd, P, I, b, active, sh);
  if (active) node_start<M, T, AOS>(nd, L, P, b);
  __syncthreads();
  int accepted = 0, iters_run = 0;
  unsigned long long mask = 0ull;
  double res[2] = {0, 0}, last_step = 0.0;
  const int Kscp = P.scp_iters;
  for (int k = 0; k < Kscp; ++k) {
    if (threadIdx.x == 0) {
      double f = 1.0;
      // the schedule tabulated at create; a warm start continues at its final penalty,
      // the one its kept ADMM state was computed at
      const int ks = (P.warm && P.warm[b]) ? Kscp - 1 : k;
      if (P.rho_fac) f = P.rho_fac[ks];
      else if (P.rho_final > 0.0 && Kscp > 1) f = pow(P.rho_final / P.rho_geo, (double)ks / (double)(Kscp - 1));
      sh.rho[0] = P.rho_eq * f; sh.rho[1] = P.rho_dyn * f; sh.rho[2] = P.rho_geo * f;
      for (int r = 0; r < 3; ++r) sh.rhof[r] = (float)sh.rho[r];
    }
    __syncthreads();
    const T re = rho_of<T>(sh, 0), rd = rho_of<T>(sh, 1), rg = rho_of<T>(sh, 2);
    const double radius = sh.radius;
    if (active) {
      if (i < N) node_jacobians<M, T, AOS>(nd, MT, I.prm, hs);
      node_setup<M, T, AOS>(nd, L, P, I, b, radius, re, rg, K);
      const bool ok = node_factor<M, T, AOS, NN>(nd, MT, L, I, K, rd, rg);
      if (!ok) atomicOr(&sh.fail, 1);
      node_reseed<M, T, AOS>(nd, L, I);
      publish_ex2<M, T, AOS>(nd, L, active, rd);
    }
    __syncthreads();
    if constexpr (GROUP) {
      // a failed factorisation in any scenario stops the whole group
      if (threadIdx.x == 0) G->mine[X.epoch & 1][0] = (double)sh.fail;
      double f[1];
      group_allreduce<1>(P, G, X, 0, f);
      if (threadIdx.x == 0) sh.fail = f[0] != 0.0;
      __syncthreads();
    }
    if (sh.fail) { if (threadIdx.x == 0) sh.status = ST_NUMERIC; iters_run++; break; }
    admm_iterations<M, T, AOS, REFINE, GROUP, REGS>(nd, MT, L, I, K, active, re, rd, rg, P.admm_iters, sh, res, G, X, P);
    ++iters_run;
    // ---- candidate (x-hat, u-hat): wide rollout, defects, cost, linear model
    W xc[NX], uc[NU], fc[NX];
    double v[6] = {0, 0, 0, 0, 0};   // cost, nl1, lin1 | dinf, step
    scp_candidate<M, T, AOS, GROUP>(nd, MT, P, I, b, active, G, sh, xc, uc, fc, v);
    bool timed_out = false;
    if (threadIdx.x == 0) timed_out = globaltimer_ns() - t0 > P.timeout_ns;
    double Jn = sh.Jn, Jc = v[0] + P.w_d * v[1], Lc = v[0] + P.w_d * v[2];
    const double Jc_own = Jc;
    if constexpr (GROUP) {
      if (threadIdx.x == 0) {
        double* m = G->mine[X.epoch & 1];
        m[0] = Jn; m[1] = Jc; m[2] = Lc; m[3] = v[3]; m[4] = v[4]; m[5] = timed_out ? 1.0 : 0.0;
      }
      double a[6];
      group_allreduce<6>(P, G, X, 3, a);
      if (threadIdx.x == 0) {
        Jn = a[0]; Jc = a[1]; Lc = a[2]; v[3] = a[3]; v[4] = a[4]; timed_out = a[5] != 0.0;
      }
    }
    if (threadIdx.x == 0) scp_decide(sh, P, Jn, Jc, Lc, Jc_own, v[3], v[4], timed_out, k, Kscp);
    __syncthreads();
    last_step = v[4];
    if (sh.accept) {
      ++accepted;
      if (k < 64) mask |= (1ull << k);
      if (active) scp_move_nominal<M, T, AOS>(nd, L, P, b, xc, uc, fc);
    }
    __syncthreads();
    if (sh.stop) break;
  }
  double w[6] = {0, 0, 0, 0, 0, 0};
  scp_finish<M, T, AOS>(nd, L, P, I, b, active, xo, uo, xout, uout, sh, w);
  if (threadIdx.x == 0) {
    bool gfail = false;
    if constexpr (GROUP) gfail = G->gfail;   // the group lost its consensus partner
    scp_report(sh, P, b, w, res, last_step, iters_run, accepted, mask, t0, gfail, stats, status_out);
  }
  __syncthreads();
  deliver_result(P, b, xout, uout, stats);
  if constexpr (GROUP) group_finish(P);
}

// Instance of a launch's CTA: instances are taken in the order given (largest
// first by default), so that the long solves of an uneven batch start in the
// first wave; a scenario group keeps its cluster's consecutive instances.
template <bool GROUP>
__device__ __forceinline__ int cta_instance(const ProblemDev& P) {
  return (GROUP || !P.order) ? (int)blockIdx.x : P.order[blockIdx.x];
}

// The fused solve for CTAs of up to MAX_THREADS threads; the compiler chooses
// the registers (up to 255: two 4-warp CTAs per SM).
template <class M, class T, bool SMEM, bool REFINE, bool GROUP = false>
__global__ void __launch_bounds__(MAX_THREADS) scp_kernel(ProblemDev P, Layout L, const double* x0, const double* u0,
                                                          double* xout, double* uout, ucn_scp_stats* stats, int* status_out) {
  scp_body<M, T, SMEM, REFINE, GROUP, true>(P, L, x0, u0, xout, uout, stats, status_out, cta_instance<GROUP>(P));
}

// The same solve for CTAs of up to 128 threads, three resident per SM (168
// registers; the ADMM state in the node records).  Each CTA runs ~1.45x longer
// than in scp_kernel, so three per SM solve ~3% more instances per unit time;
// the launcher uses it for the first round of a batch (see launch_scp_v).
constexpr int SCP3_MAX_THREADS = 128;
template <class M, class T, bool SMEM, bool REFINE>
__global__ void __launch_bounds__(SCP3_MAX_THREADS, 3) scp_kernel_3(ProblemDev P, Layout L, const double* x0,
                                                                  const double* u0, double* xout, double* uout,
                                                                  ucn_scp_stats* stats, int* status_out) {
  scp_body<M, T, SMEM, REFINE, false, false>(P, L, x0, u0, xout, uout, stats, status_out, cta_instance<false>(P));
}

}  // namespace ucn
