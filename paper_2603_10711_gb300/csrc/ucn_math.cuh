// Scalar types, dynamics models, RK4 and projections for the device path.
//
// The dynamics are written once over a scalar type S that is float, double
// or a forward-mode dual number Dual<T>; the Jacobians A_i, B_i of the RK4
// map (Sec. III-A, Eq. (2b)) are obtained by pushing one tangent direction
// at a time through the four RK4 stages.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "ucn_df.cuh"

namespace ucn {

// ------------------------------------------------------------------ dual numbers
template <class T>
struct Dual {
  T v, d;
};

template <class S> struct BaseOf { typedef S type; };
template <class T> struct BaseOf<Dual<T>> { typedef T type; };

template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
// FP32 duals divide through one correctly rounded reciprocal (the Jacobian
// passes' latency is the chain of divisions); FP64 keeps the IEEE quotient.
__device__ __forceinline__ Dual<float> operator/(Dual<float> a, Dual<float> b) {
  const float r = __frcp_rn(b.v), q = a.v * r;
  return {q, (a.d - q * b.d) * r};
}
__device__ __forceinline__ Dual<float> operator/(float a, Dual<float> b) {
  const float r = __frcp_rn(b.v), q = a * r;
  return {q, -q * b.d * r};
}
template <class T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator+(T b, Dual<T> a) { return {a.v + b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator-(T b, Dual<T> a) { return {b - a.v, -a.d}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <class T> __device__ __forceinline__ Dual<T> operator*(T b, Dual<T> a) { return {a.v * b, a.d * b}; }
template <class T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, T b) { return {a.v / b, a.d / b}; }
template <class T> __device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
  T q = a / b.v;
  return {q, -q * b.d / b.v};
}

// K tangent directions on one value (the Jacobian passes of the FP32 path): the
// value is computed once for all K; each tangent takes exactly the operations
// of Dual<T>, so the columns are those of K single-tangent passes.
template <class T, int K>
struct DualN {
  T v, d[K];
};
template <class T, int K> struct BaseOf<DualN<T, K>> { typedef T type; };
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator+(DualN<T, K> a, DualN<T, K> b) {
  DualN<T, K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = a.d[q] + b.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator-(DualN<T, K> a, DualN<T, K> b) {
  DualN<T, K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = a.d[q] - b.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator-(DualN<T, K> a) {
  DualN<T, K> r;
  r.v = -a.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = -a.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator*(DualN<T, K> a, DualN<T, K> b) {
  DualN<T, K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = a.d[q] * b.v + a.v * b.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator+(DualN<T, K> a, T b) { a.v = a.v + b; return a; }
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator+(T b, DualN<T, K> a) { a.v = a.v + b; return a; }
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator-(DualN<T, K> a, T b) { a.v = a.v - b; return a; }
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator-(T b, DualN<T, K> a) {
  DualN<T, K> r;
  r.v = b - a.v;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = -a.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator*(DualN<T, K> a, T b) {
  DualN<T, K> r;
  r.v = a.v * b;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = a.d[q] * b;
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator*(T b, DualN<T, K> a) { return a * b; }
template <class T, int K> __device__ __forceinline__ DualN<T, K> operator/(DualN<T, K> a, T b) {
  DualN<T, K> r;
  r.v = a.v / b;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = a.d[q] / b;
  return r;
}

__device__ __forceinline__ float sin_(float a) { return sinf(a); }
__device__ __forceinline__ float cos_(float a) { return cosf(a); }
__device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
__device__ __forceinline__ double sin_(double a) { return sin(a); }
__device__ __forceinline__ double cos_(double a) { return cos(a); }
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
// 1 / sqrt(a) of a Cholesky pivot: FP64 correctly rounded; FP32 by the hardware
// reciprocal square root and one Newton-Raphson step y (3 - a y^2) / 2 (within
// about one ulp; the factor feeds a refined solve), which replaces a rounded
// square root followed by a rounded divide on the factorisation's serial chain.
__device__ __forceinline__ double inv_sqrt_(double a) { return 1.0 / sqrt(a); }
__device__ __forceinline__ float inv_sqrt_(float a) {
  const float y = rsqrtf(a);
  return y * fmaf(-0.5f * a * y, y, 1.5f);
}
// Double-float: the root by one corrected step; sine and cosine (the 12-state
// quadrotor's Euler angles only) through FP64.
__device__ __forceinline__ DF sqrt_(DF a) { return df_sqrt(a); }
__device__ __forceinline__ DF sin_(DF a) { return df_from(sin(df_to_double(a))); }
__device__ __forceinline__ DF cos_(DF a) { return df_from(cos(df_to_double(a))); }
template <class T> __device__ __forceinline__ Dual<T> sin_(Dual<T> a) { return {sin_(a.v), cos_(a.v) * a.d}; }
template <class T> __device__ __forceinline__ Dual<T> cos_(Dual<T> a) { return {cos_(a.v), -sin_(a.v) * a.d}; }
template <class T> __device__ __forceinline__ Dual<T> sqrt_(Dual<T> a) {
  T s = sqrt_(a.v);
  return {s, s > T(0) ? a.d / (T(2) * s) : T(0)};
}
// DualN<float> as Dual<float> per tangent (one reciprocal per division)
template <int K> __device__ __forceinline__ DualN<float, K> operator/(DualN<float, K> a, DualN<float, K> b) {
  const float rr = __frcp_rn(b.v);
  DualN<float, K> r;
  r.v = a.v * rr;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = (a.d[q] - r.v * b.d[q]) * rr;
  return r;
}
template <int K> __device__ __forceinline__ DualN<float, K> operator/(float a, DualN<float, K> b) {
  const float rr = __frcp_rn(b.v);
  DualN<float, K> r;
  r.v = a * rr;
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = -r.v * b.d[q] * rr;
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> sin_(DualN<T, K> a) {
  const T c = cos_(a.v);
  DualN<T, K> r;
  r.v = sin_(a.v);
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = c * a.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> cos_(DualN<T, K> a) {
  const T sn = sin_(a.v);
  DualN<T, K> r;
  r.v = cos_(a.v);
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = -sn * a.d[q];
  return r;
}
template <class T, int K> __device__ __forceinline__ DualN<T, K> sqrt_(DualN<T, K> a) {
  DualN<T, K> r;
  r.v = sqrt_(a.v);
#pragma unroll
  for (int q = 0; q < K; ++q) r.d[q] = r.v > T(0) ? a.d[q] / (T(2) * r.v) : T(0);
  return r;
}

// ------------------------------------------------------------------ models
// Quadrotor, 12 states (position, velocity, ZYX Euler angles phi/theta/psi,
// body rates), 4 rotor thrusts in a "+" layout.
// prm: m, Jx, Jy, Jz, arm, km (yaw moment per unit thrust), drag, g.
struct Quad12 {
  static constexpr int NX = 12, NU = 4;
  template <class S, class P>
  __device__ static void f(const P* prm, const S* x, const S* u, S* xd) {
    typedef typename BaseOf<S>::type R;
    const R m = (R)prm[0], Jx = (R)prm[1], Jy = (R)prm[2], Jz = (R)prm[3];
    const R arm = (R)prm[4], km = (R)prm[5], cd = (R)prm[6], g = (R)prm[7];
    const S sph = sin_(x[6]), cph = cos_(x[6]);
    const S sth = sin_(x[7]), cth = cos_(x[7]);
    const S sps = sin_(x[8]), cps = cos_(x[8]);
    const S F = u[0] + u[1] + u[2] + u[3];
    // third column of R = Rz(psi) Ry(theta) Rx(phi): the body thrust axis in the world frame
    const S a0 = cph * sth * cps + sph * sps;
    const S a1 = cph * sth * sps - sph * cps;
    const S a2 = cph * cth;
    xd[0] = x[3];
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = a0 * F / m - (cd / m) * x[3];
    xd[4] = a1 * F / m - (cd / m) * x[4];
    xd[5] = a2 * F / m - g - (cd / m) * x[5];
    const S wx = x[9], wy = x[10], wz = x[11];
    const S tth = sth / cth;
    // Euler-angle rates from body rates (ZYX kinematics)
    xd[6] = wx + sph * tth * wy + cph * tth * wz;
    xd[7] = cph * wy - sph * wz;
    xd[8] = (sph * wy + cph * wz) / cth;
    // rigid-body rotation: J w' = tau - w x (J w)
    const S tx = arm * (u[1] - u[3]);
    const S ty = arm * (u[2] - u[0]);
    const S tz = km * (u[0] - u[1] + u[2] - u[3]);
    xd[9] = (tx - (Jz - Jy) * wy * wz) / Jx;
    xd[10] = (ty - (Jx - Jz) * wz * wx) / Jy;
    xd[11] = (tz - (Jy - Jx) * wx * wy) / Jz;
  }
};

// Quadrotor, 13 states (position, velocity, quaternion body-to-world scalar
// first, body rates); control = total thrust along the body z axis and three
// body torques (Sec. IV-A1).  prm as Quad12 (arm and km unused).
struct Quat13 {
  static constexpr int NX = 13, NU = 4;
  template <class S, class P>
  __device__ static void f(const P* prm, const S* x, const S* u, S* xd) {
    typedef typename BaseOf<S>::type R;
    const R m = (R)prm[0], Jx = (R)prm[1], Jy = (R)prm[2], Jz = (R)prm[3];
    const R cd = (R)prm[6], g = (R)prm[7];
    const S qw = x[6], qx = x[7], qy = x[8], qz = x[9];
    const S wx = x[10], wy = x[11], wz = x[12];
    // body z axis in the world frame, R(q) e3 (quadratic form, exact for unit q)
    const S a0 = R(2) * (qx * qz + qw * qy);
    const S a1 = R(2) * (qy * qz - qw * qx);
    const S a2 = qw * qw - qx * qx - qy * qy + qz * qz;
    const S Tm = u[0] / m;
    xd[0] = x[3];
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = a0 * Tm - (cd / m) * x[3];
    xd[4] = a1 * Tm - (cd / m) * x[4];
    xd[5] = a2 * Tm - g - (cd / m) * x[5];
    // q' = q (x) (0, w) / 2
    xd[6] = R(0.5) * (-(qx * wx) - qy * wy - qz * wz);
    xd[7] = R(0.5) * (qw * wx + qy * wz - qz * wy);
    xd[8] = R(0.5) * (qw * wy - qx * wz + qz * wx);
    xd[9] = R(0.5) * (qw * wz + qx * wy - qy * wx);
    xd[10] = (u[1] - (Jz - Jy) * wy * wz) / Jx;
    xd[11] = (u[2] - (Jx - Jz) * wz * wx) / Jy;
    xd[12] = (u[3] - (Jy - Jx) * wx * wy) / Jz;
  }
};

// Mars powered descent, 7 states: position (Up-East-North), velocity, mass;
// control = thrust vector.  prm: g (acting along -Up), alpha (mass flow per
// unit thrust), non-dimensional units.
struct Mars7 {
  static constexpr int NX = 7, NU = 3;
  // The mass rate -alpha |T|, which depends on the control alone: constant over
  // an RK4 step (the control is held), so rk4h forms it once per step.
  template <class S, class P>
  __device__ static S mass_rate(const P* prm, const S* u) {
    typedef typename BaseOf<S>::type R;
    const R alpha = (R)prm[1];
    const S Tn = sqrt_(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    return -(alpha * Tn);
  }
  template <class S, class P>
  __device__ static void f_held(const P* prm, const S* x, const S* u, const S& mdot, S* xd) {
    typedef typename BaseOf<S>::type R;
    const R g = (R)prm[0];
    const S im = R(1) / x[6];   // one division per evaluation (GB300's FP64 divide is costly)
    xd[0] = x[3];
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = u[0] * im - g;
    xd[4] = u[1] * im;
    xd[5] = u[2] * im;
    xd[6] = mdot;
  }
  template <class S, class P>
  __device__ static void f(const P* prm, const S* x, const S* u, S* xd) {
    f_held(prm, x, u, mass_rate(prm, u), xd);
  }
};

// Mars powered descent, 6-DOF, 14 states (Sec. IV-B1): mass, position
// (Up-East-North), velocity, quaternion body-to-world scalar first, body rates;
// control = thrust in the body frame (body x = thrust axis).  prm: alpha (mass
// flow per unit thrust), g (along -Up), Jx, Jy, Jz, l (the thrust acts at
// -l e_x in the body).  Non-dimensional units.
struct Mars14 {
  static constexpr int NX = 14, NU = 3;
  template <class S, class P>
  __device__ static void f(const P* prm, const S* x, const S* u, S* xd) {
    typedef typename BaseOf<S>::type R;
    const R alpha = (R)prm[0], g = (R)prm[1], Jx = (R)prm[2], Jy = (R)prm[3], Jz = (R)prm[4], l = (R)prm[5];
    const S qw = x[7], qx = x[8], qy = x[9], qz = x[10];
    const S wx = x[11], wy = x[12], wz = x[13];
    const S Tn = sqrt_(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const S im = R(1) / x[0];
    // rotation body -> world (quadratic form), applied to the body thrust
    const S c00 = qw * qw + qx * qx - qy * qy - qz * qz, c01 = R(2) * (qx * qy - qw * qz), c02 = R(2) * (qx * qz + qw * qy);
    const S c10 = R(2) * (qx * qy + qw * qz), c11 = qw * qw - qx * qx + qy * qy - qz * qz, c12 = R(2) * (qy * qz - qw * qx);
    const S c20 = R(2) * (qx * qz - qw * qy), c21 = R(2) * (qy * qz + qw * qx), c22 = qw * qw - qx * qx - qy * qy + qz * qz;
    xd[0] = -(alpha * Tn);
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = x[6];
    xd[4] = (c00 * u[0] + c01 * u[1] + c02 * u[2]) * im - g;
    xd[5] = (c10 * u[0] + c11 * u[1] + c12 * u[2]) * im;
    xd[6] = (c20 * u[0] + c21 * u[1] + c22 * u[2]) * im;
    xd[7] = R(0.5) * (-(qx * wx) - qy * wy - qz * wz);
    xd[8] = R(0.5) * (qw * wx + qy * wz - qz * wy);
    xd[9] = R(0.5) * (qw * wy - qx * wz + qz * wx);
    xd[10] = R(0.5) * (qw * wz + qx * wy - qy * wx);
    // J w' = r_T x T - w x (J w), r_T = (-l, 0, 0): r_T x T = (0, l T_z, -l T_y)
    xd[11] = (-((Jz - Jy) * wy * wz)) / Jx;
    xd[12] = (l * u[2] - (Jx - Jz) * wz * wx) / Jy;
    xd[13] = (-(l * u[1]) - (Jy - Jx) * wx * wy) / Jz;
  }
};

// a + b c in the type of a and c (one fused pass for double-float).
template <class S, class R> __device__ __forceinline__ S fma_(S a, R b, S c) { return a + b * c; }
__device__ __forceinline__ DF fma_(DF a, DF b, DF c) { return df_fma(a, b, c); }

// f with the control held over an RK4 step, as a callable x -> x-dot.  For
// the 3-DOF Mars model the control-only part (the mass rate) is formed once,
// at construction, instead of at each of the four stages: the same numbers.
template <class M, class S, class P>
struct HeldControl {
  const P* prm;
  const S* u;
  __device__ __forceinline__ HeldControl(const P* p, const S* uu) : prm(p), u(uu) {}
  __device__ __forceinline__ void operator()(const S* x, S* xd) const { M::f(prm, x, u, xd); }
};
template <class S, class P>
struct HeldControl<Mars7, S, P> {
  const P* prm;
  const S* u;
  S mdot;
  __device__ __forceinline__ HeldControl(const P* p, const S* uu) : prm(p), u(uu), mdot(Mars7::mass_rate(p, uu)) {}
  __device__ __forceinline__ void operator()(const S* x, S* xd) const { Mars7::f_held(prm, x, u, mdot, xd); }
};

// Classical fourth-order Runge-Kutta step (Eq. (1b)) with the step h and its
// multiples h/2, h/6 given in the base type R of S.
template <class M, class S, class P, class R>
__device__ __forceinline__ void rk4h(const P* prm, R h, R hh, R h6, const S* x, const S* u, S* xn) {
  constexpr int NX = M::NX;
  S k[NX], t[NX], acc[NX];
  const HeldControl<M, S, P> F(prm, u);
  F(x, k);
#pragma unroll
  for (int j = 0; j < NX; ++j) { acc[j] = k[j]; t[j] = fma_(x[j], hh, k[j]); }
  F(t, k);
#pragma unroll
  for (int j = 0; j < NX; ++j) { acc[j] = fma_(acc[j], R(2), k[j]); t[j] = fma_(x[j], hh, k[j]); }
  F(t, k);
#pragma unroll
  for (int j = 0; j < NX; ++j) { acc[j] = fma_(acc[j], R(2), k[j]); t[j] = fma_(x[j], h, k[j]); }
  F(t, k);
#pragma unroll
  for (int j = 0; j < NX; ++j) xn[j] = fma_(x[j], h6, acc[j] + k[j]);
}

template <class M, class S, class P>
__device__ __forceinline__ void rk4(const P* prm, double h_, const S* x, const S* u, S* xn) {
  typedef typename BaseOf<S>::type R;
  rk4h<M, S, P, R>(prm, (R)h_, (R)(0.5 * h_), (R)(h_ / 6.0), x, u, xn);
}

// The RK4 step h and its multiples h/2, h/6 in the arithmetic type R, rounded
// once from the FP64 step (the values rk4 forms on every call).
template <class R>
struct Step3 {
  R h, hh, h6;
};
template <class R>
__device__ __forceinline__ Step3<R> step_of(double h) {
  return {(R)h, (R)(0.5 * h), (R)(h / 6.0)};
}

// Column `dir` of [A B] = d RK4 / d(x, u) at (x, u), by one forward-mode pass.
template <class M, class T, class X, class P>
__device__ __forceinline__ void rk4_jvp(const P* prm, const Step3<T>& hs, const X* x, const X* u, int dir, T* col) {
  constexpr int NX = M::NX, NU = M::NU;
  Dual<T> xd[NX], ud[NU], out[NX];
#pragma unroll
  for (int j = 0; j < NX; ++j) xd[j] = {(T)x[j], (T)(dir == j ? 1 : 0)};
#pragma unroll
  for (int j = 0; j < NU; ++j) ud[j] = {(T)u[j], (T)(dir == NX + j ? 1 : 0)};
  rk4h<M, Dual<T>, P, T>(prm, hs.h, hs.hh, hs.h6, xd, ud, out);
#pragma unroll
  for (int j = 0; j < NX; ++j) col[j] = out[j].d;
}

// Columns dir0, dir0 + stride, ..., dir0 + (K - 1) stride of [A B] in one
// forward-mode pass (K tangents); cols[q] receives column dir0 + q stride.
template <class M, class T, int K, class X, class P>
__device__ __forceinline__ void rk4_jvpn(const P* prm, const Step3<T>& hs, const X* x, const X* u, int dir0, int stride,
                                         T (*cols)[M::NX]) {
  constexpr int NX = M::NX, NU = M::NU;
  DualN<T, K> xd[NX], ud[NU], out[NX];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    xd[j].v = (T)x[j];
#pragma unroll
    for (int q = 0; q < K; ++q) xd[j].d[q] = (T)(dir0 + q * stride == j ? 1 : 0);
  }
#pragma unroll
  for (int j = 0; j < NU; ++j) {
    ud[j].v = (T)u[j];
#pragma unroll
    for (int q = 0; q < K; ++q) ud[j].d[q] = (T)(dir0 + q * stride == NX + j ? 1 : 0);
  }
  rk4h<M, DualN<T, K>, P, T>(prm, hs.h, hs.hh, hs.h6, xd, ud, out);
#pragma unroll
  for (int j = 0; j < NX; ++j)
#pragma unroll
    for (int q = 0; q < K; ++q) cols[q][j] = out[j].d[q];
}

// ------------------------------------------------------------------ projections
// Ball {|y| <= R}: vector scaling.  FP32: the test on squares and the scale
// from one reciprocal square root (no square root, no division).
template <class T>
__device__ __forceinline__ void proj_ball3(T* y, T R) {
  if constexpr (std::is_same<T, float>::value) {
    const float n2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    if (n2 > R * R) {
      const float s = R * rsqrtf(n2);
      y[0] *= s; y[1] *= s; y[2] *= s;
    }
  } else {
    const T n = sqrt_(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    if (n > R) {
      const T s = R / n;
      y[0] *= s; y[1] *= s; y[2] *= s;
    }
  }
}

// Lorentz cone {(t, y1, y2) : |y| <= tau t}: inside -> unchanged; inside the
// polar cone (tau |y| <= -t) -> 0; otherwise onto the boundary ray.
template <class T>
__device__ __forceinline__ void proj_cone3(T* v, T tau) {
  const T t = v[0];
  const T s = sqrt_(v[1] * v[1] + v[2] * v[2]);
  if (s <= tau * t) return;
  if (tau * s <= -t) { v[0] = v[1] = v[2] = T(0); return; }
  const T ca = T(1) / sqrt_(T(1) + tau * tau), sa = tau * ca;
  const T c = t * ca + s * sa;
  v[0] = c * ca;
  const T r = c * sa / s;
  v[1] *= r;
  v[2] *= r;
}

// The same cone projection with cos / sin of the half-angle precomputed.
// FP32: the two tests on squares (tau >= 0) and one reciprocal square root.
template <class T>
__device__ __forceinline__ void proj_cone3c(T* v, T tau, T ca, T sa) {
  if constexpr (std::is_same<T, float>::value) {
    const float t = v[0], s2 = v[1] * v[1] + v[2] * v[2], t2 = t * t, tau2 = tau * tau;
    if (t >= 0.0f && s2 <= tau2 * t2) return;                              // inside
    if (t <= 0.0f && tau2 * s2 <= t2) { v[0] = v[1] = v[2] = 0.0f; return; }   // polar cone
    const float rs = rsqrtf(s2), s = s2 * rs;                               // s2 > 0 here
    const float c = t * ca + s * sa;
    v[0] = c * ca;
    const float r = c * sa * rs;
    v[1] *= r;
    v[2] *= r;
    return;
  }
  const T t = v[0];
  const T s = sqrt_(v[1] * v[1] + v[2] * v[2]);
  if (s <= tau * t) return;
  if (tau * s <= -t) { v[0] = v[1] = v[2] = T(0); return; }
  const T c = t * ca + s * sa;
  v[0] = c * ca;
  const T r = c * sa / s;
  v[1] *= r;
  v[2] *= r;
}

template <class T> __device__ __forceinline__ T clampv(T v, T lo, T hi) { return fmin(fmax(v, lo), hi); }
// max / |.| in the type of the arguments (never promoted to FP64 for floats)
__device__ __forceinline__ float maxv(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double maxv(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float absv(float a) { return fabsf(a); }
__device__ __forceinline__ double absv(double a) { return fabs(a); }
__device__ __forceinline__ float clampv(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// ------------------------------------------------------------------ warp reductions (FP64)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------ thread-block clusters
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// Cluster barrier (release on arrive, acquire on wait); every thread of every
// CTA of the cluster executes the same sequence of them.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}
// A double from the shared memory of CTA `rank` of this cluster, at the
// address that `local` has in this CTA (distributed shared memory).
__device__ __forceinline__ double ld_cluster(const double* local, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(r) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace ucn
