// Pair kernel: two threads per time node for the 3-DOF Mars model on the
// FP32 path.  Lane q in {0, 1} of a node owns the rows r = q + 2m of
// xi = (x_i, u_i) and the state rows k = q + 2m of A_i, B_i: it keeps those
// rows of A, B in registers and its rows of the cached H_i^-1 in a 52-float
// record of its own in shared memory (read by 128-bit loads, two per ADMM
// iteration), computes its rows of Steps 1-4 (Sec. III-B), and the pair
// exchanges whole vectors with one warp shuffle per row (A^T w and B^T w as
// partial sums over the lane's rows of A, B, added over the pair).  Per SCP iteration the Jacobian directions split over the pair
// (five each, one forward-mode pass), the Gram matrix of [A B] is summed over
// the pair and both lanes factor H_i; the node-level work (setup, wide
// rollout, acceptance, nominal update) maps one thread to one node.  Against
// one thread per node this halves the dependent chain of every per-node
// mat-vec and, at two CTAs per SM, gives 14 warps per SM instead of 8.
#pragma once
#include "ucn_kernels.cuh"
#include "ucn_lanes.cuh"

namespace ucn {

// CTA size cap of the pair kernel (nodes <= 112).  Registers are allocated to
// CTAs in groups of four warps, so two 7-warp CTAs per SM need <= 128 per thread.
constexpr int PAIR_MAX_THREADS = 224;
// Floats of a lane's H^-1 record: its rows of xi (5 x 10) padded to 16 bytes;
// 52 floats put the eight lanes of each quarter-warp on distinct banks for
// 128-bit loads.
constexpr int PAIR_HREC = 52;

template <class M>
struct PairRows {
  static constexpr int NX = M::NX, NU = M::NU, NN = NX + NU;
  static constexpr int R = (NN + 1) / 2;    // rows of xi per lane
  static constexpr int RA = (NX + 1) / 2;   // rows of A, B per lane (lane 1's last is empty when NX is odd)
};

// The lane's share of a node's matrices: rows q + 2m of A and B in registers
// (zero where that row does not exist) and, in shared memory at hs, full rows
// q + 2m of H^-1 (row m at hs[10 m .. 10 m + 9]).
template <class M>
struct PairMats {
  static constexpr int NX = M::NX, NU = M::NU, NN = NX + NU, R = PairRows<M>::R, RA = PairRows<M>::RA;
  static_assert(R * NN <= PAIR_HREC, "the H^-1 rows of a lane exceed its record");
  float a[RA][NX], b[RA][NU];
  float* hs;
  __device__ __forceinline__ float row(int m, int j) const { return j < NX ? a[m][j] : b[m][j - NX]; }
};

// out[m] = sum_c H^-1[row q + 2m][c] v[c] for the lane's rows, from its H^-1
// record by 128-bit loads (per row the same order of terms as sym_solve).
template <int R, int NN>
__device__ __forceinline__ void pair_hsolve(const float* hs, const float* v, float* out) {
  const float4* h4 = reinterpret_cast<const float4*>(hs);
#pragma unroll
  for (int m = 0; m < R; ++m) out[m] = 0.0f;
#pragma unroll
  for (int k = 0; k < (R * NN + 3) / 4; ++k) {
    const float4 hv = h4[k];
    const float e[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int idx = 4 * k + t;
      if (idx < R * NN) out[idx / NN] += e[t] * v[idx % NN];
    }
  }
}

// A packed symmetric matrix in registers (assembly and factorisation).
template <int n>
struct PackedH {
  mutable float hp[n * (n + 1) / 2];
  __device__ __forceinline__ float& H(int k) const { return hp[k]; }
};

// v <- v(lane 0) + v(lane 1) in both lanes (float addition is commutative, so
// both lanes hold the same bits).  Every lane of the warp calls it.
template <int n>
__device__ __forceinline__ void pair_sum(float* v) {
#pragma unroll
  for (int k = 0; k < n; ++k) v[k] += __shfl_xor_sync(WARP_ALL, v[k], 1);
}

// full[r], r < n, from the lanes' own rows own[m] = row q + 2m.  Every lane of
// the warp calls it.
template <int n>
__device__ __forceinline__ void pair_gather(const float* own, float* full, int q) {
#pragma unroll
  for (int m = 0; m < (n + 1) / 2; ++m) {
    const float o = __shfl_xor_sync(WARP_ALL, own[m], 1);
    if (2 * m < n) full[2 * m] = q ? o : own[m];
    if (2 * m + 1 < n) full[2 * m + 1] = q ? own[m] : o;
  }
}

// Entry m of a compile-time-indexed full vector for this lane's row q + 2m.
template <int n>
__device__ __forceinline__ float own_of(const float* v, int m, int q) {
  const float e = v[2 * m < n ? 2 * m : n - 1];
  const float o = v[2 * m + 1 < n ? 2 * m + 1 : n - 1];
  return q ? (2 * m + 1 < n ? o : 0.0f) : (2 * m < n ? e : 0.0f);
}

// A_i, B_i (Eq. (2b)): lane q differentiates the RK4 map along directions
// q KD .. q KD + KD - 1 in one forward-mode pass, then the pair swaps columns so
// that each lane holds its rows.  Every lane of the warp calls it; has_u:
// the node has a control (else its rows are zero).
template <class M>
__device__ __forceinline__ void pair_jacobians(const Node<float, true>& nd, PairMats<M>& PM, const float* prm,
                                               const Step3<float>& hs, int q, bool has_u) {
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU, RA = PairRows<M>::RA, KD = (NN + 1) / 2;
  float xt[NX], ut[NU];
#pragma unroll
  for (int j = 0; j < NX; ++j) xt[j] = has_u ? wide_to<float>(nd.dat(Rec<M>::Xbar, j)) : 0.0f;
#pragma unroll
  for (int j = 0; j < NU; ++j) ut[j] = has_u ? wide_to<float>(nd.dat(Rec<M>::Ubar, j)) : 1.0f;
  float cols[KD][NX];
  rk4_jvpn<M, float, KD>(prm, hs, xt, ut, q * KD, 1, cols);
#pragma unroll
  for (int m = 0; m < RA; ++m) {
#pragma unroll
    for (int c = 0; c < KD; ++c) {
      // rows 2m (lane 0's) and 2m + 1 (lane 1's) of this lane's column c
      const float r0 = (2 * m < NX) ? cols[c][2 * m < NX ? 2 * m : 0] : 0.0f;
      const float r1 = (2 * m + 1 < NX) ? cols[c][2 * m + 1 < NX ? 2 * m + 1 : 0] : 0.0f;
      const float mine = q ? r1 : r0;
      const float recv = __shfl_xor_sync(WARP_ALL, q ? r0 : r1, 1);
      // lane 0 holds columns c (its own) and KD + c (the partner's); lane 1 the reverse
      const float lo = has_u ? (q ? recv : mine) : 0.0f, hi = has_u ? (q ? mine : recv) : 0.0f;
      if (c < NX) PM.a[m][c < NX ? c : 0] = lo;
      else if (c < NN) PM.b[m][c - NX < NU ? c - NX : 0] = lo;
      if (KD + c < NX) PM.a[m][KD + c < NX ? KD + c : 0] = hi;
      else if (KD + c < NN) PM.b[m][KD + c - NX < NU && KD + c >= NX ? KD + c - NX : 0] = hi;
    }
  }
}

// The node's cost gradient (deviations) and the diagonal of H_i without its
// A/B and mirror Gram terms -- the values node_setup puts in NodeConst --
// for every row (hd) and for this lane's rows (kq, khd).
template <class M>
__device__ __forceinline__ void pair_consts(const Node<float, true>& nd, const Inst<float>& I, int q, float re,
                                            float rg, float* kq, float* khd, float* hd) {
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU, R = PairRows<M>::R;
  typedef CB<M> C;
  const DF* cb = nd.c;
  const int i = nd.i, N = nd.N;
  const bool term = (i == N);
  const bool cost = term || I.run_cost;
  float qf[NN];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    const DF w = term ? cb[C::QNd + j] : cb[C::Qd + j];
    if (cost) {
      DF gq = df_mul(df_sub(nd.dat(Rec<M>::Xbar, j), cb[C::Xref + j]), w);
      if (term) gq = df_add(gq, cb[C::QN + j]);
      qf[j] = df_to_float(gq);
    } else {
      qf[j] = 0.0f;
    }
    hd[j] = df_to_float(w) + rg + (i > 0 ? re : 0.0f);
  }
#pragma unroll
  for (int j = 0; j < NU; ++j) {
    qf[NX + j] = 0.0f;
    hd[NX + j] = 1.0f;
    if (!term) {
      const DF w = cb[C::Rd + j];
      qf[NX + j] = I.run_cost ? df_to_float(df_mul(df_sub(nd.dat(Rec<M>::Ubar, j), cb[C::Uref + j]), w)) : 0.0f;
      hd[NX + j] = df_to_float(w) + rg;
    }
  }
#pragma unroll
  for (int m = 0; m < R; ++m) {
    kq[m] = own_of<NN>(qf, m, q);
    khd[m] = own_of<NN>(hd, m, q);
  }
}

// H_i of Eq. (4) with the Mars mirror Gram terms (glide-slope cone on the
// position, thrust ball and linearised lower bound on the control), as
// node_factor assembles it, from the pair's summed Gram matrix of [A B];
// factored and inverted by both lanes, each keeping its rows of H^-1.  Every
// lane of the warp calls it.
template <class M>
__device__ __forceinline__ bool pair_factor(const Node<float, true>& nd, PairMats<M>& PM, const Layout& L,
                                            const Inst<float>& I, const float* hd, float rd, float rg, int q,
                                            bool active) {
  constexpr int NX = M::NX, NN = NX + M::NU, R = PairRows<M>::R, RA = PairRows<M>::RA;
  const bool term = nd.i == nd.N;
  PackedH<NN> H;
#pragma unroll
  for (int r = 0; r < NN; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < RA; ++m) acc += PM.row(m, r) * PM.row(m, c);
      H.hp[pk(r, c)] = acc;
    }
  pair_sum<NN*(NN + 1) / 2>(H.hp);
  float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f;
  if (active && !term && I.half) { n0 = nd.at(L.oMd, 0); n1 = nd.at(L.oMd, 1); n2 = nd.at(L.oMd, 2); }
  const float nv[3] = {n0, n1, n2};
#pragma unroll
  for (int r = 0; r < NN; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      const float G = H.hp[pk(r, c)];
      float h = 0.0f;
      if (r < NX) {                 // H11
        if (r == c) h = hd[r];
        if (!term) h += rd * G;
        if (r < 3 && r == c && I.cone) h += rg;
      } else if (c < NX) {          // H21 (zero at node N)
        h = term ? 0.0f : rd * G;
      } else {                      // H22 (identity at node N)
        const int rr = r - NX, cc = c - NX;
        if (rr == cc) h = hd[r];
        if (!term) h += rd * G;
        if (rr < 3 && cc < 3 && !term) {
          if (rr == cc && I.ball) h += rg;
          if (I.half) h += rg * nv[rr < 3 ? rr : 0] * nv[cc < 3 ? cc : 0];
        }
      }
      H.hp[pk(r, c)] = h;
    }
  const bool ok = factor_invert_packed<float, NN>(H);
  if (active) {
    float4* h4 = reinterpret_cast<float4*>(PM.hs);
#pragma unroll
    for (int k = 0; k < PAIR_HREC / 4; ++k) {
      float e[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int idx = 4 * k + t, m = idx / NN, c = idx % NN;
        const int r0 = 2 * m < NN ? 2 * m : NN - 1, r1 = 2 * m + 1 < NN ? 2 * m + 1 : NN - 1;
        const float ev = H.hp[r0 >= c ? pk(r0, c) : pk(c, r0)], ov = H.hp[r1 >= c ? pk(r1, c) : pk(c, r1)];
        e[t] = idx < R * NN ? (q ? (2 * m + 1 < NN ? ov : 0.0f) : ev) : 0.0f;
      }
      h4[k] = make_float4(e[0], e[1], e[2], e[3]);
    }
  }
  return ok;
}

// One iteration of Steps 1-4 (Sec. III-B) with two threads per node; every
// thread of the CTA calls it (inactive nodes with zero data: the shuffles need
// whole warps).  The LAST instance also sums the residual norms (as
// admm_iteration).  3-DOF Mars sets: glide-slope cone (lane 0), thrust ball and
// linearised lower bound (lane 1).
template <class M, bool REFINE, bool LAST>
__device__ __forceinline__ void admm_iteration_pair(const Node<float, true>& nd, const PairMats<M>& PM,
                                                    const Layout& L, const Inst<float>& I, const float* kq,
                                                    const float* khd, bool active, int q, float re, float rd,
                                                    float rg, float irg, float ired, DF& rp, DF& rdl, GroupX& X) {
  static_assert(std::is_same<M, Mars7>::value, "the pair kernel carries the 3-DOF Mars sets");
  typedef Rec<M> RC;
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU, R = PairRows<M>::R, RA = PairRows<M>::RA;
  const int i = nd.i, N = nd.N;
  const bool has_u = active && i < N;
  float xo[R], xf[NN];
  // ---- Step 1: g_i (own rows), H_i xi = g_i by the cached inverse (+ one refinement)
  {
    // A^T w, B^T w with w_k = mu_{i+1} + rho_dyn (z_{i+1} - c_i): partial sums over the
    // lane's rows k, then over the pair
    float pw[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) pw[j] = 0.0f;
#pragma unroll
    for (int m = 0; m < RA; ++m) {
      const int k = q + 2 * m;
      const float w = (has_u && k < NX) ? nd.nb(RC::Ex2, k, i + 1) - rd * nd.at(RC::C, k) : 0.0f;
#pragma unroll
      for (int j = 0; j < NX; ++j) pw[j] += PM.a[m][j] * w;
#pragma unroll
      for (int j = 0; j < NU; ++j) pw[NX + j] += PM.b[m][j] * w;
    }
    pair_sum<NN>(pw);
    float g[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + 2 * m;
      float v = 0.0f;
      if (active) {
        if (r < NX) {
          v = -kq[m] + rg * nd.at(RC::Xh, r) - nd.at(RC::Nux, r);
          if (i > 0) v += re * nd.at(RC::Z, r) - nd.at(RC::Lam, r);
          v += own_of<NN>(pw, m, q);
          if (I.cone && r < 3) v += rg * nd.at(L.oS, r) - nd.at(L.oNus, r);
        } else if (i < N) {
          const int j = r - NX;
          v = -kq[m] + own_of<NN>(pw, m, q) + rg * nd.at(RC::Uh, j) - nd.at(RC::Nuu, j);
          if (I.ball) v += rg * nd.at(L.oS, 3 + j) - nd.at(L.oNus, 3 + j);
          if (I.half) v += nd.at(L.oMd, j) * (rg * nd.at(L.oS, 6) - nd.at(L.oNus, 6));
        }
      }
      g[m] = v;
    }
    float gf[NN];
    pair_gather<NN>(g, gf, q);
    if (active) pair_hsolve<R, NN>(PM.hs, gf, xo);
    else
#pragma unroll
      for (int m = 0; m < R; ++m) xo[m] = 0.0f;
    if constexpr (REFINE) {
      // residual g - H xi, H applied from A, B, the diagonals and the mirror Gram terms
      pair_gather<NN>(xo, xf, q);
      float pv[NN];
#pragma unroll
      for (int j = 0; j < NN; ++j) pv[j] = 0.0f;
#pragma unroll
      for (int m = 0; m < RA; ++m) {
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < NX; ++c) acc += PM.a[m][c] * xf[c];
#pragma unroll
        for (int c = 0; c < NU; ++c) acc += PM.b[m][c] * xf[NX + c];
        const float v = has_u ? rd * acc : 0.0f;
#pragma unroll
        for (int j = 0; j < NX; ++j) pv[j] += PM.a[m][j] * v;
#pragma unroll
        for (int j = 0; j < NU; ++j) pv[NX + j] += PM.b[m][j] * v;
      }
      pair_sum<NN>(pv);
      const float nu_dot = (has_u && I.half)
                               ? rg * (nd.at(L.oMd, 0) * xf[NX] + nd.at(L.oMd, 1) * xf[NX + 1] + nd.at(L.oMd, 2) * xf[NX + 2])
                               : 0.0f;
      float res[R];
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = q + 2 * m;
        float hx = khd[m] * xo[m];
        if (has_u) hx += own_of<NN>(pv, m, q);
        if (r < 3 && I.cone) hx += rg * xo[m];
        if (r >= NX && has_u) {
          if (I.ball) hx += rg * xo[m];
          if (I.half) hx += nd.at(L.oMd, r - NX) * nu_dot;
        }
        res[m] = g[m] - hx;
      }
      float rf[NN];
      pair_gather<NN>(res, rf, q);
      if (active) {
        float dx[R];
        pair_hsolve<R, NN>(PM.hs, rf, dx);
#pragma unroll
        for (int m = 0; m < R; ++m) xo[m] += dx[m];
      }
    }
    pair_gather<NN>(xo, xf, q);
    if (active) {
      // linearised propagation d_dyn,i = A x + B u + c_i (the lane's rows), published to node i+1
      if (has_u) {
#pragma unroll
        for (int m = 0; m < RA; ++m) {
          const int k = q + 2 * m;
          if (k < NX) {
            float acc = nd.at(RC::C, k);
#pragma unroll
            for (int c = 0; c < NX; ++c) acc += PM.a[m][c] * xf[c];
#pragma unroll
            for (int c = 0; c < NU; ++c) acc += PM.b[m][c] * xf[NX + c];
            nd.at(RC::Ex1, k) = acc;
          }
        }
      }
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = q + 2 * m;
        if (r < NX) nd.at(RC::X, r) = xo[m];
        else if (has_u) nd.at(RC::U, r - NX) = xo[m];
      }
    }
  }
  // Step 3 before Step 2 (disjoint variables; both read only this iteration's xi),
  // between the arrival on the split barrier and the wait for the left neighbour's Ex1
  split_barrier_arrive(X.bar);
  float svo[R], msv[NN];   // dual-residual terms: own rows | mirror terms of all rows (LAST)
#pragma unroll
  for (int m = 0; m < R; ++m) svo[m] = 0.0f;
#pragma unroll
  for (int j = 0; j < NN; ++j) msv[j] = 0.0f;
  if (active) {
    // ---- Step 3: box projections (Eq. (7)) and Step 4 for nu_x, nu_u (own rows)
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + 2 * m;
      if (r < NX) {
        const float nux = nd.at(RC::Nux, r);
        const float xh = clampv(xo[m] + nux * irg, nd.at(RC::Xlo, r), nd.at(RC::Xhi, r));
        if (LAST) { svo[m] += rg * (xh - nd.at(RC::Xh, r)); acc_sq_diff(rp, xo[m], xh); }
        nd.at(RC::Xh, r) = xh;
        nd.at(RC::Nux, r) = nux + rg * (xo[m] - xh);
      } else if (i < N) {
        const int j = r - NX;
        const float nuu = nd.at(RC::Nuu, j);
        const float uh = clampv(xo[m] + nuu * irg, nd.at(RC::Ulo, j), nd.at(RC::Uhi, j));
        if (LAST) { svo[m] += rg * (uh - nd.at(RC::Uh, j)); acc_sq_diff(rp, xo[m], uh); }
        nd.at(RC::Uh, j) = uh;
        nd.at(RC::Nuu, j) = nuu + rg * (xo[m] - uh);
      }
    }
    // mirror sets: the glide-slope cone on lane 0, the thrust sets on lane 1
    if (q == 0) {
      if (I.cone) {
        float v[3], xb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          xb[k] = nd.at(L.oMd, 4 + k);
          v[k] = xb[k] + xf[k] + nd.at(L.oNus, k) * irg;
        }
        proj_cone3c(v, I.tau, I.ca, I.sa);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float s = v[k] - xb[k];
          const float so = nd.at(L.oS, k);
          nd.at(L.oS, k) = s;
          nd.at(L.oNus, k) += rg * (xf[k] - s);
          if (LAST) { msv[k] += rg * (s - so); acc_sq_diff(rp, xf[k], s); }
        }
      }
    } else if (i < N) {
      float ub[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) ub[k] = nd.at(L.oMd, 7 + k);
      if (I.ball) {
        float v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = ub[k] + xf[NX + k] + nd.at(L.oNus, 3 + k) * irg;
        proj_ball3(v, I.tmax);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float s = v[k] - ub[k];
          const float so = nd.at(L.oS, 3 + k);
          nd.at(L.oS, 3 + k) = s;
          nd.at(L.oNus, 3 + k) += rg * (xf[NX + k] - s);
          if (LAST) { msv[NX + k] += rg * (s - so); acc_sq_diff(rp, xf[NX + k], s); }
        }
      }
      if (I.half) {
        const float n0 = nd.at(L.oMd, 0), n1 = nd.at(L.oMd, 1), n2 = nd.at(L.oMd, 2), bd = nd.at(L.oMd, 3);
        const float y = n0 * xf[NX] + n1 * xf[NX + 1] + n2 * xf[NX + 2];
        const float so = nd.at(L.oS, 6);
        const float s = maxv(bd, y + nd.at(L.oNus, 6) * irg);
        nd.at(L.oS, 6) = s;
        nd.at(L.oNus, 6) += rg * (y - s);
        if (LAST) {
          const float ds = rg * (s - so);
          msv[NX] += n0 * ds; msv[NX + 1] += n1 * ds; msv[NX + 2] += n2 * ds;
          acc_sq_diff(rp, y, s);
        }
      }
    }
  }
  split_barrier_wait(X.bar, X.ph);
  float dz[R];
#pragma unroll
  for (int m = 0; m < R; ++m) dz[m] = 0.0f;
  if (active && i >= 1) {
    // ---- Step 2: dynamic consensus, Eq. (5), then its duals (Step 4), own state rows
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + 2 * m;
      if (r < NX) {
        const float dd = nd.nb(RC::Ex1, r, i - 1);
        const float zo = nd.at(RC::Z, r);
        const float lam = nd.at(RC::Lam, r), mu = nd.at(RC::Mu, r);
        const float z = (re * xo[m] + lam + rd * dd - mu) * ired;
        nd.at(RC::Z, r) = z;
        nd.at(RC::Lam, r) = lam + re * (xo[m] - z);
        nd.at(RC::Mu, r) = mu + rd * (z - dd);
        dz[m] = z - zo;
        if (LAST) {
          svo[m] += re * dz[m];
          acc_sq_diff(rp, xo[m], z);
          acc_sq_diff(rp, z, dd);
        }
      }
    }
  }
  if constexpr (LAST) {
    pair_sum<NN>(msv);
#pragma unroll
    for (int m = 0; m < R; ++m) svo[m] += own_of<NN>(msv, m, q);
    // dual residual: rho_dyn (z_{i+1,new} - z_{i+1,old}) of the right neighbour through A^T, B^T
    __syncthreads();
    if (active && i >= 1) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = q + 2 * m;
        if (r < NX) nd.at(RC::Ex1, r) = rd * dz[m];
      }
    }
    __syncthreads();
    float pe[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) pe[j] = 0.0f;
#pragma unroll
    for (int m = 0; m < RA; ++m) {
      const int k = q + 2 * m;
      const float e = (has_u && k < NX) ? nd.nb(RC::Ex1, k, i + 1) : 0.0f;
#pragma unroll
      for (int j = 0; j < NX; ++j) pe[j] += PM.a[m][j] * e;
#pragma unroll
      for (int j = 0; j < NU; ++j) pe[NX + j] += PM.b[m][j] * e;
    }
    pair_sum<NN>(pe);
    if (active) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int r = q + 2 * m;
        if (r < NX || i < N) acc_sq(rdl, svo[m] + (has_u ? own_of<NN>(pe, m, q) : 0.0f));
      }
    }
  }
  if (active && i >= 1) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = q + 2 * m;
      if (r < NX) nd.at(RC::Ex2, r) = nd.at(RC::Mu, r) + rd * nd.at(RC::Z, r);
    }
  }
  __syncthreads();
}

template <class M, bool REFINE>
__device__ __forceinline__ void admm_iterations_pair(const Node<float, true>& nd, const PairMats<M>& PM,
                                                     const Layout& L, const Inst<float>& I, const float* kq,
                                                     const float* khd, bool active, int q, float re, float rd,
                                                     float rg, int iters, InstShared& sh, double* res, GroupX& X) {
  const float irg = 1.0f / rg, ired = 1.0f / (re + rd);
  DF rp, rdl;   // residual sums (double-float; see acc_sq_diff)
  for (int it = 0; it + 1 < iters; ++it)
    admm_iteration_pair<M, REFINE, false>(nd, PM, L, I, kq, khd, active, q, re, rd, rg, irg, ired, rp, rdl, X);
  admm_iteration_pair<M, REFINE, true>(nd, PM, L, I, kq, khd, active, q, re, rd, rg, irg, ired, rp, rdl, X);
  reduce_residuals(sh, rp, rdl, res);
}

// The candidate of an SCP iteration (as scp_candidate): the node-level part
// (trajectory, wide rollout, defects, cost, step) on the dense mapping `ndd`,
// the linear-model defects on the pair's rows of A, B; CTA totals in v.
template <class M>
__device__ void pair_candidate(const Node<float, true>& ndd, bool dact, const Node<float, true>& nd,
                               const PairMats<M>& PM, bool has_u, int q, const ProblemDev& P, const Inst<float>& I,
                               int b, InstShared& sh, DF* xc, DF* uc, DF* fc, double* v) {
  typedef Rec<M> RC;
  constexpr int NX = M::NX, NU = M::NU, RA = PairRows<M>::RA;
  const int i = ndd.i, N = ndd.N;
  if (dact) {
    for (int j = 0; j < NX; ++j) { xc[j] = wide_add(ndd.dat(RC::Xbar, j), ndd.at(RC::Xh, j)); ndd.dat(RC::Xc, j) = xc[j]; }
    for (int j = 0; j < NU; ++j) uc[j] = (i < N) ? wide_add(ndd.dat(RC::Ubar, j), ndd.at(RC::Uh, j)) : DF();
  }
  __syncthreads();
  DF vs[3] = {DF(), DF(), DF()};   // cost, nl1, lin1
  float dinf = 0.0f, st = 0.0f, lin1 = 0.0f;
  if (dact) {
    vs[0] = node_cost<M, float, true>(ndd, P, I, b, i, N, xc, uc);
    for (int j = 0; j < NX; ++j) st = maxv(st, absv(ndd.at(RC::Xh, j)));
    if (i < N) {
      for (int j = 0; j < NU; ++j) st = maxv(st, absv(ndd.at(RC::Uh, j)));
      rk4_wide<M, float, true>(ndd, P, b, xc, uc, fc);
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        fc[r] = fc[r] - ndd.dnb(RC::Xc, r, i + 1);
        vs[1] = vs[1] + wide_abs(fc[r]);
        dinf = maxv(dinf, wide_abs_round(fc[r]));
      }
    }
  }
  if (has_u) {
    const int in = nd.i;
    float xh[NX], uh[NU];
#pragma unroll
    for (int c = 0; c < NX; ++c) xh[c] = nd.at(RC::Xh, c);
#pragma unroll
    for (int c = 0; c < NU; ++c) uh[c] = nd.at(RC::Uh, c);
#pragma unroll
    for (int m = 0; m < RA; ++m) {
      const int k = q + 2 * m;
      if (k < NX) {
        float lin = nd.at(RC::C, k) - nd.nb(RC::Xh, k, in + 1);
#pragma unroll
        for (int c = 0; c < NX; ++c) lin += PM.a[m][c] * xh[c];
#pragma unroll
        for (int c = 0; c < NU; ++c) lin += PM.b[m][c] * uh[c];
        lin1 += absv(lin);
      }
    }
  }
  vs[2] = df_from(lin1);
  float mx[2] = {dinf, st};
  block_reduce_df(sh, vs, 3, mx, 2, v);
}

// The fused SCP solve (as scp_kernel) with two threads per node: 3-DOF Mars,
// FP32 path, node records in shared memory.
template <class M, bool REFINE>
__global__ void __launch_bounds__(PAIR_MAX_THREADS, 2) scp_kernel_pair(ProblemDev P, Layout L, const double* x0,
                                                                       const double* u0, double* xout, double* uout,
                                                                       ucn_scp_stats* stats, int* status_out) {
  typedef DF W;
  constexpr int NX = M::NX, NU = M::NU, R = PairRows<M>::R, NN = NX + NU;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ InstShared sh;
  GroupX X{0u, 0, 0};
  const int b = P.order ? P.order[blockIdx.x] : (int)blockIdx.x;
  const int q = (int)threadIdx.x & 1;
  Node<float, true> nd = make_node_at<float, true>(P, L, smem, b, (int)threadIdx.x >> 1);
  Node<float, true> ndd = make_node<float, true>(P, L, smem, b);   // one thread per node
  const int i = nd.i, N = nd.N;
  const bool active = i <= N, has_u = active && i < N;
  const bool dact = ndd.i <= N;
  const long long xo = P.xoff[b], uo = P.uoff[b];
  const Step3<float> hs = step_of<float>(P.dt[b]);   // the RK4 step in FP32, once per launch
  const unsigned long long t0 = globaltimer_ns();
  const Inst<float> I = make_inst<M, float>(P, b);
  NodeConst<M, float> Kd;   // node_setup's constants on the dense mapping (not used there)
  PairMats<M> PM;
  PM.hs = reinterpret_cast<float*>(smem + L.oPH) + (long long)threadIdx.x * PAIR_HREC;
  float kq[R], khd[R];
#pragma unroll
  for (int m = 0; m < R; ++m) { kq[m] = 0.0f; khd[m] = 0.0f; }
  if (threadIdx.x == 0) {
    sh.fail = 0; sh.status = ST_OK; sh.radius = P.tr_init; sh.stop = 0;
    split_barrier_init(sh.xbar, blockDim.x);
  }
  X.bar = sh.xbar;
  stage_consts<M, float, true>(ndd, P, b);
  if (dact) load_nominal<M, float, true>(ndd, L, x0, u0, xo, uo);
  __syncthreads();
  flag_bad_inputs<M>(P, b, x0, u0, xo, uo, sh);
  scp_start<M, float, true>(ndd, P, I, b, dact, sh);
  if (dact) node_start<M, float, true>(ndd, L, P, b);
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
    const float re = sh.rhof[0], rd = sh.rhof[1], rg = sh.rhof[2];
    const double radius = sh.radius;
    pair_jacobians<M>(nd, PM, I.prm, hs, q, has_u);
    if (dact) {
      node_setup<M, float, true>(ndd, L, P, I, b, radius, re, rg, Kd);
      node_reseed<M, float, true>(ndd, L, I);
      publish_ex2<M, float, true>(ndd, L, true, rd);
    }
    __syncthreads();
    float hd[NN];
    if (active) pair_consts<M>(nd, I, q, re, rg, kq, khd, hd);
    else
#pragma unroll
      for (int j = 0; j < NN; ++j) hd[j] = 1.0f;
    const bool ok = pair_factor<M>(nd, PM, L, I, hd, rd, rg, q, active);
    if (active && !ok) atomicOr(&sh.fail, 1);
    __syncthreads();
    if (sh.fail) { if (threadIdx.x == 0) sh.status = ST_NUMERIC; iters_run++; break; }
    admm_iterations_pair<M, REFINE>(nd, PM, L, I, kq, khd, active, q, re, rd, rg, P.admm_iters, sh, res, X);
    ++iters_run;
    // ---- candidate (x-hat, u-hat): wide rollout, defects, cost, linear model
    W xc[NX], uc[NU], fc[NX];
    double v[6] = {0, 0, 0, 0, 0};   // cost, nl1, lin1 | dinf, step
    pair_candidate<M>(ndd, dact, nd, PM, has_u, q, P, I, b, sh, xc, uc, fc, v);
    bool timed_out = false;
    if (threadIdx.x == 0) timed_out = globaltimer_ns() - t0 > P.timeout_ns;
    const double Jn = sh.Jn, Jc = v[0] + P.w_d * v[1], Lc = v[0] + P.w_d * v[2];
    if (threadIdx.x == 0) scp_decide(sh, P, Jn, Jc, Lc, Jc, v[3], v[4], timed_out, k, Kscp);
    __syncthreads();
    last_step = v[4];
    if (sh.accept) {
      ++accepted;
      if (k < 64) mask |= (1ull << k);
      if (dact) scp_move_nominal<M, float, true>(ndd, L, P, b, xc, uc, fc);
    }
    __syncthreads();
    if (sh.stop) break;
  }
  double w[6] = {0, 0, 0, 0, 0, 0};
  scp_finish<M, float, true>(ndd, L, P, I, b, dact, xo, uo, xout, uout, sh, w);
  if (threadIdx.x == 0)
    scp_report(sh, P, b, w, res, last_step, iters_run, accepted, mask, t0, false, stats, status_out);
  __syncthreads();
  deliver_result(P, b, xout, uout, stats);
}

}  // namespace ucn
