// Lane-parallel fused SCP kernel: TPN consecutive threads of a warp share one
// time node.  Lane q owns the rows r of xi = (x_i, u_i) with r % TPN == q
// (x rows q, q+TPN, ..., control rows NX+q, NX+q+TPN, ...), computes their
// parts of Steps 1-4 (Sec. III-B), and the lanes of a node exchange whole
// vectors with warp shuffles.  Compared with one thread per node this divides
// the dependent chain of the per-node mat-vecs by TPN and multiplies the
// resident warps by TPN -- the one-thread kernel of a 16-row node runs 1-2
// warps per scheduler and is latency-bound.  The per-SCP-iteration work
// (assembly and factorisation, the wide rollout, acceptance) maps one thread
// to one node again; the Jacobian directions are split over the lanes.
#pragma once
#include "ucn_kernels.cuh"

namespace ucn {

constexpr int LANES_MAX_THREADS = 512;   // CTA size cap of the lane kernel
// CTA size cap of its wide-register variant: __launch_bounds__(384, 1) lets a
// thread hold 168 registers (65,536 / 384, allocation granularity), which the
// 16-row node state needs to stay out of local memory; the launcher takes it
// whenever it keeps as many CTAs per SM resident as the other variant.
constexpr int LANES_WIDE_THREADS = 384;
constexpr unsigned WARP_ALL = 0xffffffffu;

template <class M, int TPN>
struct LaneRows {
  static constexpr int NX = M::NX, NU = M::NU, NN = NX + NU;
  static_assert(NX % TPN == 0 && NU % TPN == 0, "rows must split evenly over the lanes");
  static constexpr int RX = NX / TPN, RU = NU / TPN, R = RX + RU;
};

// full[r] for every row r of a node from the lanes' own rows (shuffles inside
// the TPN-lane segment; every thread of the warp must call it).
template <class M, int TPN, class T>
__device__ __forceinline__ void lanes_gather(const T* own, T* full) {
  using LR = LaneRows<M, TPN>;
#pragma unroll
  for (int s = 0; s < TPN; ++s) {
#pragma unroll
    for (int m = 0; m < LR::RX; ++m) full[s + TPN * m] = __shfl_sync(WARP_ALL, own[m], s, TPN);
#pragma unroll
    for (int m = 0; m < LR::RU; ++m) full[LR::NX + s + TPN * m] = __shfl_sync(WARP_ALL, own[LR::RX + m], s, TPN);
  }
}

// The x-rows only (NX entries).
template <class M, int TPN, class T>
__device__ __forceinline__ void lanes_gather_x(const T* own, T* full) {
  using LR = LaneRows<M, TPN>;
#pragma unroll
  for (int s = 0; s < TPN; ++s)
#pragma unroll
    for (int m = 0; m < LR::RX; ++m) full[s + TPN * m] = __shfl_sync(WARP_ALL, own[m], s, TPN);
}

// Sum of v[0..n) over the TPN lanes of a node (butterfly).
template <int TPN, int n, class T>
__device__ __forceinline__ void lanes_allreduce(T* v) {
#pragma unroll
  for (int o = 1; o < TPN; o <<= 1)
#pragma unroll
    for (int k = 0; k < n; ++k) v[k] += __shfl_xor_sync(WARP_ALL, v[k], o, TPN);
}

// Row r of xi owned by lane q as its m-th row.
template <class M, int TPN>
__device__ __forceinline__ int own_row(int q, int m) {
  using LR = LaneRows<M, TPN>;
  return m < LR::RX ? q + TPN * m : LR::NX + q + TPN * (m - LR::RX);
}

// The lane's rows of the cached H^-1: registers for FP32 (loaded once per SCP
// iteration), the packed record in shared memory for FP64.
template <class M, class T, int TPN, bool REG>
struct LaneH;
template <class M, class T, int TPN>
struct LaneH<M, T, TPN, true> {
  static constexpr int NN = M::NX + M::NU, R = LaneRows<M, TPN>::R;
  T h[R][NN];
  template <class MS>
  __device__ __forceinline__ void load(const MS& MT, int q, bool active) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int r = own_row<M, TPN>(q, m);
#pragma unroll
      for (int c = 0; c < NN; ++c) h[m][c] = active ? MT.H(r >= c ? pk(r, c) : pk(c, r)) : T(0);
    }
  }
  template <class MS>
  __device__ __forceinline__ T get(const MS&, int, int m, int c) const { return h[m][c]; }
};
template <class M, class T, int TPN>
struct LaneH<M, T, TPN, false> {
  int rb[LaneRows<M, TPN>::R];   // packed offset of the start of each own row
  template <class MS>
  __device__ __forceinline__ void load(const MS&, int q, bool) {
#pragma unroll
    for (int m = 0; m < LaneRows<M, TPN>::R; ++m) { const int r = own_row<M, TPN>(q, m); rb[m] = r * (r + 1) / 2; }
  }
  template <class MS>
  __device__ __forceinline__ T get(const MS& MT, int q, int m, int c) const {
    const int r = own_row<M, TPN>(q, m);
    return MT.H(r >= c ? rb[m] + c : pk(c, 0) + r);
  }
};

// A_i, B_i (Eq. (2b)): the NN forward-mode directions split over the lanes.
template <class M, class T, bool AOS, int TPN, class MS>
__device__ __forceinline__ void lanes_jacobians(const Node<T, AOS>& nd, const MS& MT, const T* prm, const Step3<T>& hs,
                                                int q) {
  constexpr int NX = M::NX, NU = M::NU;
  typename Node<T, AOS>::W xb[NX], ub[NU];
  read_nominal<M, T, AOS>(nd, true, xb, ub);
  T xt[NX], ut[NU];
#pragma unroll
  for (int j = 0; j < NX; ++j) xt[j] = wide_to<T>(xb[j]);
#pragma unroll
  for (int j = 0; j < NU; ++j) ut[j] = wide_to<T>(ub[j]);
  if constexpr (std::is_same<T, float>::value) {
    // FP32: the lane's directions two per pass (q, q + TPN), (q + 2 TPN, q + 3 TPN), ...
    for (int dir = q; dir < NX + NU; dir += 2 * TPN) {
      const int dir1 = dir + TPN;
      T cols[2][NX];
      if (dir1 < NX + NU) rk4_jvpn<M, T, 2>(prm, hs, xt, ut, dir, TPN, cols);
      else rk4_jvp<M, T>(prm, hs, xt, ut, dir, cols[0]);
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        if (dir < NX) MT.A(r, dir) = cols[0][r];
        else MT.B(r, dir - NX) = cols[0][r];
        if (dir1 < NX + NU) {
          if (dir1 < NX) MT.A(r, dir1) = cols[1][r];
          else MT.B(r, dir1 - NX) = cols[1][r];
        }
      }
    }
  } else {
    for (int dir = q; dir < NX + NU; dir += TPN) {
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

// The lane's rows of the cost gradient (q_i, r_i) in deviations and of the
// diagonal of H_i without its A/B and mirror Gram terms (the same numbers as
// node_setup's NodeConst, for the own rows only).
template <class M, class T, bool AOS, int TPN>
__device__ __forceinline__ void lanes_consts(const Node<T, AOS>& nd, const ProblemDev& P, int b, int q, T re, T rg,
                                             T* kq, T* khd) {
  using LR = LaneRows<M, TPN>;
  constexpr int NX = M::NX, NU = M::NU;
  const int i = nd.i, N = nd.N;
  const bool term = (i == N);
  if constexpr (IsDF<T>::value) {
    typedef CB<M> C;
    const DF* cb = nd.c;
#pragma unroll
    for (int m = 0; m < LR::RX; ++m) {
      const int j = q + TPN * m;
      const DF w = term ? cb[C::QNd + j] : cb[C::Qd + j];
      DF gq = df_mul(df_sub(nd.dat(Rec<M>::Xbar, j), cb[C::Xref + j]), w);
      if (term) gq = df_add(gq, cb[C::QN + j]);
      kq[m] = df_to_float(gq);
      khd[m] = df_to_float(w) + rg + (i > 0 ? re : T(0));
    }
#pragma unroll
    for (int m = 0; m < LR::RU; ++m) {
      const int j = q + TPN * m;
      if (term) {
        kq[LR::RX + m] = T(0);
        khd[LR::RX + m] = T(1);
      } else {
        const DF w = cb[C::Rd + j];
        kq[LR::RX + m] = df_to_float(df_mul(df_sub(nd.dat(Rec<M>::Ubar, j), cb[C::Uref + j]), w));
        khd[LR::RX + m] = df_to_float(w) + rg;
      }
    }
    return;
  } else {
#pragma unroll
  for (int m = 0; m < LR::RX; ++m) {
    const int j = q + TPN * m;
    const double w = term ? P.QNd[b * NX + j] : P.Qd[b * NX + j];
    kq[m] = (T)(w * (nd.dat(Rec<M>::Xbar, j) - P.xref[b * NX + j]) + (term ? P.qN[b * NX + j] : 0.0));
    khd[m] = (T)w + rg + (i > 0 ? re : T(0));
  }
#pragma unroll
  for (int m = 0; m < LR::RU; ++m) {
    const int j = q + TPN * m;
    if (term) {
      kq[LR::RX + m] = T(0);
      khd[LR::RX + m] = T(1);
    } else {
      kq[LR::RX + m] = (T)(P.Rd[b * NU + j] * (nd.dat(Rec<M>::Ubar, j) - P.uref[b * NU + j]));
      khd[LR::RX + m] = (T)P.Rd[b * NU + j] + rg;
    }
  }
  }
}

// One iteration of Steps 1-4 over the CTA's instance, lane-parallel.  Every
// thread of the CTA calls it (inactive nodes with zero data: the shuffles
// need whole warps).  Quadrotor mirror sets (linearised obstacles) only.
template <class M, class T, bool AOS, bool REFINE, bool LAST, bool GROUP, int TPN, class MS, class HR>
__device__ __forceinline__ void admm_iteration_lanes(const Node<T, AOS>& nd, const MS& MT, const HR& H, const Layout& L,
                                                     const Inst<T>& I, const T* kq, const T* khd, bool active, int q,
                                                     T re, T rd, T rg, T irg, T ired, typename WideOf<T>::type& rp,
                                               typename WideOf<T>::type& rdl,
                                                     GroupShared* G, GroupX& X, const ProblemDev& P) {
  static_assert(IsQuad<M>::value, "the lane kernel carries the quadrotor's mirror sets");
  using LR = LaneRows<M, TPN>;
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU, RX = LR::RX, RU = LR::RU, R = LR::R;
  const int i = nd.i, N = nd.N;
  const bool hasU = active && i < N;
  T xo[R];      // own rows of xi
  T xf[NN];     // all rows of xi (after the final gather)
  // ---- Step 1: g_i (own rows), H_i xi = g_i by the cached inverse (+ one refinement)
  {
    T w[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) w[k] = hasU ? nd.nb(Rec<M>::Ex2, k, i + 1) - rd * nd.at(Rec<M>::C, k) : T(0);
    T g[R];
#pragma unroll
    for (int m = 0; m < RX; ++m) {
      const int j = q + TPN * m;
      T v = T(0);
      if (active) {
        v = -kq[m] + rg * nd.at(Rec<M>::Xh, j) - nd.at(Rec<M>::Nux, j);
        if (i > 0) v += re * nd.at(Rec<M>::Z, j) - nd.at(Rec<M>::Lam, j);
        if (hasU) {
          T acc = T(0);
#pragma unroll
          for (int k = 0; k < NX; ++k) acc += MT.A(k, j) * w[k];
          v += acc;
        }
        if (m == 0 && j < 3)
          for (int o = 0; o < I.nobs; ++o) v += nd.at(L.oMd, ObsStride<T>::value * o + j) * (rg * nd.at(L.oS, o) - nd.at(L.oNus, o));
      }
      g[m] = v;
    }
#pragma unroll
    for (int m = 0; m < RU; ++m) {
      const int j = q + TPN * m;
      T v = T(0);
      if (hasU) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) acc += MT.B(k, j) * w[k];
        v = -kq[RX + m] + acc + rg * nd.at(Rec<M>::Uh, j) - nd.at(Rec<M>::Nuu, j);
      }
      g[RX + m] = v;
    }
    T gf[NN];
    lanes_gather<M, TPN>(g, gf);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      T t = T(0);
      if (active) {
#pragma unroll
        for (int c = 0; c < NN; ++c) t += H.get(MT, q, m, c) * gf[c];
      }
      xo[m] = t;
    }
    if constexpr (REFINE) {
      // residual g - H xi with H applied from A, B, the diagonals and the mirror Gram terms
      lanes_gather<M, TPN>(xo, xf);
      T vo[RX];
#pragma unroll
      for (int m = 0; m < RX; ++m) {
        const int k = q + TPN * m;
        T acc = T(0);
        if (hasU) {
#pragma unroll
          for (int c = 0; c < NX; ++c) acc += MT.A(k, c) * xf[c];
#pragma unroll
          for (int c = 0; c < NU; ++c) acc += MT.B(k, c) * xf[NX + c];
        }
        vo[m] = rd * acc;
      }
      T vf[NX];
      lanes_gather_x<M, TPN>(vo, vf);
      T res[R];
#pragma unroll
      for (int m = 0; m < RX; ++m) {
        const int j = q + TPN * m;
        T hx = khd[m] * xo[m];
        if (hasU) {
#pragma unroll
          for (int k = 0; k < NX; ++k) hx += MT.A(k, j) * vf[k];
        }
        if (active && m == 0 && j < 3)
          for (int o = 0; o < I.nobs; ++o) {
            const T n0 = nd.at(L.oMd, ObsStride<T>::value * o), n1 = nd.at(L.oMd, ObsStride<T>::value * o + 1), n2 = nd.at(L.oMd, ObsStride<T>::value * o + 2);
            hx += nd.at(L.oMd, ObsStride<T>::value * o + j) * (rg * (n0 * xf[0] + n1 * xf[1] + n2 * xf[2]));
          }
        res[m] = g[m] - hx;
      }
#pragma unroll
      for (int m = 0; m < RU; ++m) {
        const int j = q + TPN * m;
        T hx = khd[RX + m] * xo[RX + m];
        if (hasU) {
#pragma unroll
          for (int k = 0; k < NX; ++k) hx += MT.B(k, j) * vf[k];
        }
        res[RX + m] = g[RX + m] - hx;
      }
      T rf[NN];
      lanes_gather<M, TPN>(res, rf);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        T t = T(0);
        if (active) {
#pragma unroll
          for (int c = 0; c < NN; ++c) t += H.get(MT, q, m, c) * rf[c];
        }
        xo[m] += t;
      }
    }
    lanes_gather<M, TPN>(xo, xf);
    if (active) {
      // linearised propagation d_dyn,i = A x + B u + c_i, published to node i+1
      if (hasU) {
#pragma unroll
        for (int m = 0; m < RX; ++m) {
          const int k = q + TPN * m;
          T acc = nd.at(Rec<M>::C, k);
#pragma unroll
          for (int c = 0; c < NX; ++c) acc += MT.A(k, c) * xf[c];
#pragma unroll
          for (int c = 0; c < NU; ++c) acc += MT.B(k, c) * xf[NX + c];
          nd.at(Rec<M>::Ex1, k) = acc;
        }
      }
#pragma unroll
      for (int m = 0; m < RX; ++m) nd.at(Rec<M>::X, q + TPN * m) = xo[m];
      if (hasU) {
#pragma unroll
        for (int m = 0; m < RU; ++m) nd.at(Rec<M>::U, q + TPN * m) = xo[RX + m];
      }
    }
  }
  // Step 3 before Step 2 (disjoint variables, both read only this iteration's
  // xi): between the arrival on the split barrier and the wait for the left
  // neighbour's Ex1
  if constexpr (GROUP) __syncthreads();   // groups: their exchange follows Step 2 on a plain barrier
  else split_barrier_arrive(X.bar);
  T dz[RX];
  T sv[R];
#pragma unroll
  for (int m = 0; m < R; ++m) sv[m] = T(0);
#pragma unroll
  for (int m = 0; m < RX; ++m) dz[m] = T(0);
  T msv[3] = {T(0), T(0), T(0)};
  if (active) {
    // ---- Step 3: projections onto the boxes (Eq. (7)) and Step 4 for nu_x, nu_u
#pragma unroll
    for (int m = 0; m < RX; ++m) {
      const int j = q + TPN * m;
      const T nux = nd.at(Rec<M>::Nux, j);
      const T xh = clampv(xo[m] + nux * irg, nd.at(Rec<M>::Xlo, j), nd.at(Rec<M>::Xhi, j));
      if (LAST) { sv[m] += rg * (xh - nd.at(Rec<M>::Xh, j)); acc_sq_diff(rp, xo[m], xh); }
      nd.at(Rec<M>::Xh, j) = xh;
      nd.at(Rec<M>::Nux, j) = nux + rg * (xo[m] - xh);
    }
    if (i < N) {
#pragma unroll
      for (int m = 0; m < RU; ++m) {
        const int j = q + TPN * m;
        const T nuu = nd.at(Rec<M>::Nuu, j);
        if constexpr (GROUP) {
          if (i == 0) {   // sum of arguments | max of lower bounds | max of -upper bounds
            const double ub = wide_to_double(nd.dat(Rec<M>::Ubar, j));
            double* mm = G->mine[X.epoch & 1];
            mm[j] = ub + (double)(xo[RX + m] + nuu * irg);
            mm[NU + j] = ub + (double)nd.at(Rec<M>::Ulo, j);
            mm[2 * NU + j] = -(ub + (double)nd.at(Rec<M>::Uhi, j));
            continue;
          }
        }
        const T uh = clampv(xo[RX + m] + nuu * irg, nd.at(Rec<M>::Ulo, j), nd.at(Rec<M>::Uhi, j));
        if (LAST) {
          sv[RX + m] += rg * (uh - nd.at(Rec<M>::Uh, j));
          acc_sq_diff(rp, xo[RX + m], uh);
        }
        nd.at(Rec<M>::Uh, j) = uh;
        nd.at(Rec<M>::Nuu, j) = nuu + rg * (xo[RX + m] - uh);
      }
    }
    // linearised obstacles (mirror half-spaces on the position), split over the lanes
    for (int o = q; o < I.nobs; o += TPN) {
      const T n0 = nd.at(L.oMd, ObsStride<T>::value * o), n1 = nd.at(L.oMd, ObsStride<T>::value * o + 1), n2 = nd.at(L.oMd, ObsStride<T>::value * o + 2);
      const T bd = nd.at(L.oMd, ObsStride<T>::value * o + 3);
      const T y = n0 * xf[0] + n1 * xf[1] + n2 * xf[2];
      const T so = nd.at(L.oS, o);
      const T s = maxv(bd, y + nd.at(L.oNus, o) * irg);
      nd.at(L.oS, o) = s;
      nd.at(L.oNus, o) += rg * (y - s);
      if (LAST) {
        const T ds = rg * (s - so);
        msv[0] += n0 * ds; msv[1] += n1 * ds; msv[2] += n2 * ds;
        acc_sq_diff(rp, y, s);
      }
    }
  }
  if constexpr (!GROUP) split_barrier_wait(X.bar, X.ph);
  if (active) {
    // ---- Step 2: dynamic consensus, Eq. (5), then its duals (Step 4)
    if (i >= 1) {
#pragma unroll
      for (int m = 0; m < RX; ++m) {
        const int j = q + TPN * m;
        const T dd = nd.nb(Rec<M>::Ex1, j, i - 1);
        const T zo = nd.at(Rec<M>::Z, j);
        const T lam = nd.at(Rec<M>::Lam, j), mu = nd.at(Rec<M>::Mu, j);
        const T z = (re * xo[m] + lam + rd * dd - mu) * ired;
        nd.at(Rec<M>::Z, j) = z;
        nd.at(Rec<M>::Lam, j) = lam + re * (xo[m] - z);
        nd.at(Rec<M>::Mu, j) = mu + rd * (z - dd);
        dz[m] = z - zo;
        if (LAST) {
          sv[m] += re * dz[m];
          acc_sq_diff(rp, xo[m], z); acc_sq_diff(rp, z, dd);
        }
      }
    }
  }
  if constexpr (GROUP) {
    double tot[3 * NU];
#pragma unroll
    for (int j = 0; j < 3 * NU; ++j) tot[j] = 0.0;
    group_allreduce<3 * NU>(P, G, X, NU, tot);
#pragma unroll
    for (int j = 0; j < 3 * NU; ++j) tot[j] = __shfl_sync(WARP_ALL, tot[j], 0, TPN);
    if (active && i == 0 && i < N) {
#pragma unroll
      for (int m = 0; m < RU; ++m) {
        const int j = q + TPN * m;
        const double v = fmin(fmax(tot[j] / (double)P.group, tot[NU + j]), -tot[2 * NU + j]);
        G->u0[j] = v;
        const T uh = (T)(v - wide_to_double(nd.dat(Rec<M>::Ubar, j)));
        const T nuu = nd.at(Rec<M>::Nuu, j);
        if (LAST) {
          sv[RX + m] += rg * (uh - nd.at(Rec<M>::Uh, j));
          acc_sq_diff(rp, xo[RX + m], uh);
        }
        nd.at(Rec<M>::Uh, j) = uh;
        nd.at(Rec<M>::Nuu, j) = nuu + rg * (xo[RX + m] - uh);
      }
    }
  }
  if constexpr (LAST) {
    // the obstacle terms of the dual residual belong to the position rows
    lanes_allreduce<TPN, 3>(msv);
    if (q < 3) sv[0] += msv[q == 0 ? 0 : (q == 1 ? 1 : 2)];
    // dual residual needs rho_dyn (z_{i+1,new} - z_{i+1,old}) from the right neighbour
    __syncthreads();
    if (active && i >= 1) {
#pragma unroll
      for (int m = 0; m < RX; ++m) nd.at(Rec<M>::Ex1, q + TPN * m) = rd * dz[m];
    }
    __syncthreads();
    if (hasU) {
      T e[NX];
#pragma unroll
      for (int k = 0; k < NX; ++k) e[k] = nd.nb(Rec<M>::Ex1, k, i + 1);
#pragma unroll
      for (int m = 0; m < RX; ++m) {
        const int j = q + TPN * m;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) acc += MT.A(k, j) * e[k];
        sv[m] += acc;
      }
#pragma unroll
      for (int m = 0; m < RU; ++m) {
        const int j = q + TPN * m;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) acc += MT.B(k, j) * e[k];
        sv[RX + m] += acc;
      }
    }
    if (active) {
#pragma unroll
      for (int m = 0; m < R; ++m)
        if (m < RX || i < N) acc_sq(rdl, sv[m]);
    }
  }
  if (active && i >= 1) {
#pragma unroll
    for (int m = 0; m < RX; ++m) {
      const int j = q + TPN * m;
      nd.at(Rec<M>::Ex2, j) = nd.at(Rec<M>::Mu, j) + rd * nd.at(Rec<M>::Z, j);
    }
  }
  __syncthreads();
}

template <class M, class T, bool AOS, bool REFINE, bool GROUP, int TPN, class MS, class HR>
__device__ __forceinline__ void admm_iterations_lanes(const Node<T, AOS>& nd, const MS& MT, const HR& H, const Layout& L,
                                                      const Inst<T>& I, const T* kq, const T* khd, bool active, int q,
                                                      T re, T rd, T rg, int iters, InstShared& sh, double* res,
                                                      GroupShared* G, GroupX& X, const ProblemDev& P) {
  const T irg = T(1) / rg, ired = T(1) / (re + rd);
  typename WideOf<T>::type rp{}, rdl{};   // residual sums in the wide type (FP64 or double-float)
  for (int it = 0; it + 1 < iters; ++it)
    admm_iteration_lanes<M, T, AOS, REFINE, false, GROUP, TPN>(nd, MT, H, L, I, kq, khd, active, q, re, rd, rg, irg,
                                                               ired, rp, rdl, G, X, P);
  admm_iteration_lanes<M, T, AOS, REFINE, true, GROUP, TPN>(nd, MT, H, L, I, kq, khd, active, q, re, rd, rg, irg, ired,
                                                            rp, rdl, G, X, P);
  // squared norms (the root is taken once, when they are reported)
  reduce_residuals(sh, rp, rdl, res);
}

// Node view of node `i` (the lane kernel maps TPN threads to a node).
template <class T, bool SMEM>
__device__ __forceinline__ Node<T, SMEM> make_node_at(const ProblemDev& P, const Layout& L, unsigned char* smem, int b,
                                                      int i) {
  Node<T, SMEM> nd = make_node<T, SMEM>(P, L, smem, b);
  nd.i = i;
  return nd;
}

// The fused SCP solve (as scp_kernel) with TPN lanes per node: the body of the
// two kernels below.
template <class M, class T, bool SMEM, bool REFINE, bool GROUP, int TPN>
__device__ __forceinline__ void scp_lanes_body(const ProblemDev& P, const Layout& L, const double* x0,
                                               const double* u0, double* xout, double* uout, ucn_scp_stats* stats,
                                               int* status_out, const int b) {
  using LR = LaneRows<M, TPN>;
  constexpr int NX = M::NX, NU = M::NU, NN = NX + NU, R = LR::R;
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
  const int q = (int)threadIdx.x % TPN;
  Node<T, AOS> nd = make_node_at<T, SMEM>(P, L, smem, b, (int)threadIdx.x / TPN);
  SmemMats<M, T, AOS> MT;
  init_mats<M, T, AOS>(MT, nd, L);
  LaneH<M, T, TPN, std::is_same<T, float>::value> H;
  const int i = nd.i, N = nd.N;
  const bool active = i <= N;
  // The per-SCP-iteration work (nominal, assembly and factorisation, the wide
  // rollout and acceptance, the nominal update) maps one thread to one node, so
  // that its warps run full -- the FP64 plain path's FP64 pipe charges a warp
  // instruction whatever its active lanes.
  Node<T, AOS> ndd = make_node<T, SMEM>(P, L, smem, b);
  SmemMats<M, T, AOS> MTd;
  init_mats<M, T, AOS>(MTd, ndd, L);
  const int id = ndd.i;
  const bool dact = id <= N;
  typedef typename Node<T, AOS>::W W;
  const long long xo = P.xoff[b], uo = P.uoff[b];
  const Step3<T> hs = step_of<T>(P.dt[b]);   // the RK4 step in T, once per launch
  const unsigned long long t0 = globaltimer_ns();
  const Inst<T> I = make_inst<M, T>(P, b);
  NodeConst<M, T> K;
  T kq[R], khd[R];
#pragma unroll
  for (int m = 0; m < R; ++m) { kq[m] = T(0); khd[m] = T(0); }
  if (threadIdx.x == 0) {
    sh.fail = 0; sh.status = ST_OK; sh.radius = P.tr_init; sh.stop = 0;
    split_barrier_init(sh.xbar, blockDim.x);
  }
  X.bar = sh.xbar;
  stage_consts<M, T, AOS>(ndd, P, b);
  if (dact) load_nominal<M, T, AOS>(ndd, L, x0, u0, xo, uo);
  __syncthreads();
  flag_bad_inputs<M>(P, b, x0, u0, xo, uo, sh);
  scp_start<M, T, AOS>(ndd, P, I, b, dact, sh);
  if (dact) node_start<M, T, AOS>(ndd, L, P, b);
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
    if (active && i < N) lanes_jacobians<M, T, AOS, TPN>(nd, MT, I.prm, hs, q);
    if (active) lanes_consts<M, T, AOS, TPN>(nd, P, b, q, re, rg, kq, khd);
    __syncthreads();
    if (dact) {
      node_setup<M, T, AOS>(ndd, L, P, I, b, radius, re, rg, K);
      const bool ok = node_factor<M, T, AOS, NN>(ndd, MTd, L, I, K, rd, rg);
      if (!ok) atomicOr(&sh.fail, 1);
      node_reseed<M, T, AOS>(ndd, L, I);
      publish_ex2<M, T, AOS>(ndd, L, true, rd);
    }
    __syncthreads();
    H.load(MT, q, active);
    if constexpr (GROUP) {
      if (threadIdx.x == 0) G->mine[X.epoch & 1][0] = (double)sh.fail;
      double f[1];
      group_allreduce<1>(P, G, X, 0, f);
      if (threadIdx.x == 0) sh.fail = f[0] != 0.0;
      __syncthreads();
    }
    if (sh.fail) { if (threadIdx.x == 0) sh.status = ST_NUMERIC; iters_run++; break; }
    admm_iterations_lanes<M, T, AOS, REFINE, GROUP, TPN>(nd, MT, H, L, I, kq, khd, active, q, re, rd, rg, P.admm_iters,
                                                         sh, res, G, X, P);
    ++iters_run;
    // ---- candidate (x-hat, u-hat): wide rollout, defects, cost, linear model (dense mapping)
    W xc[NX], uc[NU], fc[NX];
    double v[6] = {0, 0, 0, 0, 0};
    scp_candidate<M, T, AOS, GROUP>(ndd, MTd, P, I, b, dact, G, sh, xc, uc, fc, v);
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
      if (dact) scp_move_nominal<M, T, AOS>(ndd, L, P, b, xc, uc, fc);
    }
    __syncthreads();
    if (sh.stop) break;
  }
  double w[6] = {0, 0, 0, 0, 0, 0};
  scp_finish<M, T, AOS>(ndd, L, P, I, b, dact, xo, uo, xout, uout, sh, w);
  if (threadIdx.x == 0) {
    bool gfail = false;
    if constexpr (GROUP) gfail = G->gfail;   // the group lost its consensus partner
    scp_report(sh, P, b, w, res, last_step, iters_run, accepted, mask, t0, gfail, stats, status_out);
  }
  __syncthreads();
  deliver_result(P, b, xout, uout, stats);
  if constexpr (GROUP) group_finish(P);
}

// CTAs of up to 512 threads; the compiler chooses the registers (128 at most).
template <class M, class T, bool SMEM, bool REFINE, bool GROUP, int TPN>
__global__ void __launch_bounds__(LANES_MAX_THREADS) scp_kernel_lanes(ProblemDev P, Layout L, const double* x0,
                                                                      const double* u0, double* xout, double* uout,
                                                                      ucn_scp_stats* stats, int* status_out) {
  scp_lanes_body<M, T, SMEM, REFINE, GROUP, TPN>(P, L, x0, u0, xout, uout, stats, status_out, cta_instance<GROUP>(P));
}

// CTAs of up to 384 threads, one resident per SM guaranteed its registers (168).
template <class M, class T, bool SMEM, bool REFINE, bool GROUP, int TPN>
__global__ void __launch_bounds__(LANES_WIDE_THREADS, 1) scp_kernel_lanes_wide(ProblemDev P, Layout L,
                                                                               const double* x0, const double* u0,
                                                                               double* xout, double* uout,
                                                                               ucn_scp_stats* stats, int* status_out) {
  scp_lanes_body<M, T, SMEM, REFINE, GROUP, TPN>(P, L, x0, u0, xout, uout, stats, status_out, cta_instance<GROUP>(P));
}

// The kernel of register class MAXT (LANES_WIDE_THREADS or LANES_MAX_THREADS).
template <class M, class T, bool SMEM, bool REFINE, bool GROUP, int TPN, int MAXT>
constexpr auto lanes_kernel() {
  if constexpr (MAXT == LANES_WIDE_THREADS) return scp_kernel_lanes_wide<M, T, SMEM, REFINE, GROUP, TPN>;
  else return scp_kernel_lanes<M, T, SMEM, REFINE, GROUP, TPN>;
}

}  // namespace ucn
