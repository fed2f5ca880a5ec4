// FP64 CPU oracle for GPU-native SCP + consensus ADMM (arXiv 2603.10711).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// reference that the CUDA path is checked against.  Only the tests, the smoke
// check and the benchmark's CPU-baseline leg may load it; the library never
// does.  It shares no code, header or helper with the CUDA path.
//
// Everything is FP64 and written as plain loops in the order the paper
// states the method:
//   * dynamics f and its RK4 discretisation (Eq. (1b), "4th-order Runge-Kutta")
//   * linearisation A_i, B_i, d_i about the nominal (Eq. (2b), Sec. III-A)
//     by the RK4 variational equations with hand-derived f_x, f_u
//   * the convex QP of Eq. (2) with trust-region boxes (Eq. (2c))
//   * consensus ADMM on the augmented Lagrangian of Eq. (3):
//       Step 1  per-node KKT solve H_i xi_i = g_i, H_i from Eq. (4), unpivoted
//               Cholesky factor cached for the whole ADMM call
//       Step 2  closed-form dynamic consensus, Eq. (5)
//       Step 3  projections (clamp, Eq. (7); ball, cone, half-space)
//       Step 4  dual ascent, Eq. (8) and its analogues
//   * the SCP loop with a trust-region acceptance test (the paper omits this
//     logic, Sec. III-A, and points to standard texts; the reading used here
//     is a ratio test on an l1 merit function).
//
// Readings where the paper is silent (all listed in the design notes):
//   - Non-box sets (linearised obstacle half-spaces, thrust ball, thrust lower
//     bound, glide-slope cone) each get their own mirror variable s_j = G_j xi
//     with dual nu_j and penalty rho_geo, exactly like x-hat and u-hat.  This
//     keeps the two-block structure of the convergence remark (Sec. III-B).
//   - x-hat_0 = x_init and the S-selected components of x-hat_N = x_target;
//     the boundary conditions Eq. (1c) enter as the sets X_0 and X_N.
//   - Node N carries no control; H_N = Q_N + (rho_geo + rho_eq) I + mirrors.
//   - ADMM is warm-started across SCP iterations; at each new SCP iteration
//     every mirror is re-projected from the current x-hat/u-hat with the new
//     G_j, duals kept.
//   - Duals are kept unscaled (Eq. (3) form), so a rho change needs no rescale.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fopenmp -shared -fPIC
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { MODEL_QUAD12 = 1, MODEL_MARS7 = 2, MODEL_QUAT13 = 3, MODEL_MARS14 = 4 };
enum { BLK_NONE = -1, BLK_HALF = 0, BLK_BALL = 1, BLK_CONE = 2 };
enum { ST_OK = 0, ST_NUMERIC = 4, ST_NOTCONV = 5 };

// ============================================================= models
// Quadrotor, 12 states: p(3), v(3), eta = (phi, theta, psi) ZYX Euler angles,
// omega(3) body rates.  u = four rotor thrusts in a "+" layout.
// params: m, Jx, Jy, Jz, arm l, yaw coefficient km, linear drag cd, g.
//   p' = v
//   v' = R(eta) e3 (f1+f2+f3+f4)/m - g e3 - (cd/m) v,  R = Rz(psi) Ry(theta) Rx(phi)
//   eta' = W(phi,theta) omega   (ZYX Euler-rate kinematics)
//   omega' = J^-1 (tau - omega x J omega),
//   tau = (l (f2 - f4), l (f3 - f1), km (f1 - f2 + f3 - f4))
template <class S>
void quad_f(const double* prm, const S* x, const S* u, S* xd) {
  const double m = prm[0], Jx = prm[1], Jy = prm[2], Jz = prm[3];
  const double l = prm[4], km = prm[5], cd = prm[6], g = prm[7];
  S sphi = sin(x[6]), cphi = cos(x[6]);
  S sth = sin(x[7]), cth = cos(x[7]);
  S sps = sin(x[8]), cps = cos(x[8]);
  S F = u[0] + u[1] + u[2] + u[3];
  S a0 = cphi * sth * cps + sphi * sps;
  S a1 = cphi * sth * sps - sphi * cps;
  S a2 = cphi * cth;
  for (int k = 0; k < 3; ++k) xd[k] = x[3 + k];
  xd[3] = a0 * F / m - (cd / m) * x[3];
  xd[4] = a1 * F / m - (cd / m) * x[4];
  xd[5] = a2 * F / m - g - (cd / m) * x[5];
  S wx = x[9], wy = x[10], wz = x[11];
  S tth = sth / cth;
  xd[6] = wx + sphi * tth * wy + cphi * tth * wz;
  xd[7] = cphi * wy - sphi * wz;
  xd[8] = (sphi * wy + cphi * wz) / cth;
  S tx = l * (u[1] - u[3]);
  S ty = l * (u[2] - u[0]);
  S tz = km * (u[0] - u[1] + u[2] - u[3]);
  xd[9] = (tx - (Jz - Jy) * wy * wz) / Jx;
  xd[10] = (ty - (Jx - Jz) * wz * wx) / Jy;
  xd[11] = (tz - (Jy - Jx) * wx * wy) / Jz;
}

// Mars powered descent, 7 states: r(3) Up-East-North, v(3), mass m; u = thrust T(3).
// params: g (magnitude, acting along -Up), alpha (mass flow per unit thrust).
//   r' = v,  v' = T/m + (-g, 0, 0),  m' = -alpha |T|
template <class S>
void mars_f(const double* prm, const S* x, const S* u, S* xd) {
  const double g = prm[0], alpha = prm[1];
  S Tn = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int k = 0; k < 3; ++k) xd[k] = x[3 + k];
  xd[3] = u[0] / x[6] - g;
  xd[4] = u[1] / x[6];
  xd[5] = u[2] / x[6];
  xd[6] = -alpha * Tn;
}

// Quadrotor, 13 states (Sec. IV-A1): r(3), v(3), unit quaternion q = (qw, qx,
// qy, qz) body-to-world, omega(3) body rates; u = (T, tau_x, tau_y, tau_z) total
// thrust along the body z axis and body torques.  params as quad_f (arm and km
// unused).  Newton-Euler:
//   r' = v
//   v' = (T/m) R(q) e3 - g e3 - (cd/m) v,
//        R(q) e3 = (2(qx qz + qw qy), 2(qy qz - qw qx), qw^2 - qx^2 - qy^2 + qz^2)
//   q' = 1/2 q (x) (0, omega)          (Hamilton product)
//   omega' = J^-1 (tau - omega x J omega)
// The quaternion is integrated as four states (no renormalisation); R(q) e3 is
// the quadratic form of the rotation, exact for unit q.
template <class S>
void quat_f(const double* prm, const S* x, const S* u, S* xd) {
  const double m = prm[0], Jx = prm[1], Jy = prm[2], Jz = prm[3], cd = prm[6], g = prm[7];
  const S qw = x[6], qx = x[7], qy = x[8], qz = x[9];
  const S wx = x[10], wy = x[11], wz = x[12];
  const S T = u[0];
  const S a0 = 2.0 * (qx * qz + qw * qy);
  const S a1 = 2.0 * (qy * qz - qw * qx);
  const S a2 = qw * qw - qx * qx - qy * qy + qz * qz;
  for (int k = 0; k < 3; ++k) xd[k] = x[3 + k];
  xd[3] = a0 * T / m - (cd / m) * x[3];
  xd[4] = a1 * T / m - (cd / m) * x[4];
  xd[5] = a2 * T / m - g - (cd / m) * x[5];
  xd[6] = 0.5 * (-qx * wx - qy * wy - qz * wz);
  xd[7] = 0.5 * (qw * wx + qy * wz - qz * wy);
  xd[8] = 0.5 * (qw * wy - qx * wz + qz * wx);
  xd[9] = 0.5 * (qw * wz + qx * wy - qy * wx);
  xd[10] = (u[1] - (Jz - Jy) * wy * wz) / Jx;
  xd[11] = (u[2] - (Jx - Jz) * wz * wx) / Jy;
  xd[12] = (u[3] - (Jy - Jx) * wx * wy) / Jz;
}

// Mars powered descent, 6-DOF, 14 states (Sec. IV-B1): mass m, position r
// (Up-East-North), velocity v, quaternion q = (qw, qx, qy, qz) body-to-world
// scalar first, body rates omega; u = thrust T in the body frame (body x is
// the thrust axis).  params: alpha (mass flow per unit thrust), g (along -Up),
// Jx, Jy, Jz (diagonal inertia), l (the thrust acts at -l e_x in the body).
//   m' = -alpha |T|
//   r' = v
//   v' = C(q) T / m + (-g, 0, 0)
//   q' = 1/2 q (x) (0, omega)
//   omega' = J^-1 (r_T x T - omega x J omega),  r_T = (-l, 0, 0)
// C(q) is the quadratic form of the rotation matrix (exact for unit q).
template <class S>
void quat_rot(const S* q, S C[3][3]) {
  const S w = q[0], a = q[1], b = q[2], c = q[3];
  C[0][0] = w * w + a * a - b * b - c * c; C[0][1] = 2.0 * (a * b - w * c); C[0][2] = 2.0 * (a * c + w * b);
  C[1][0] = 2.0 * (a * b + w * c); C[1][1] = w * w - a * a + b * b - c * c; C[1][2] = 2.0 * (b * c - w * a);
  C[2][0] = 2.0 * (a * c - w * b); C[2][1] = 2.0 * (b * c + w * a); C[2][2] = w * w - a * a - b * b + c * c;
}

template <class S>
void mars6_f(const double* prm, const S* x, const S* u, S* xd) {
  const double alpha = prm[0], g = prm[1], Jx = prm[2], Jy = prm[3], Jz = prm[4], l = prm[5];
  const S m = x[0];
  const S* q = &x[7];
  const S wx = x[11], wy = x[12], wz = x[13];
  S C[3][3];
  quat_rot<S>(q, C);
  const S Tn = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  xd[0] = -alpha * Tn;
  for (int k = 0; k < 3; ++k) xd[1 + k] = x[4 + k];
  for (int k = 0; k < 3; ++k) xd[4 + k] = (C[k][0] * u[0] + C[k][1] * u[1] + C[k][2] * u[2]) / m;
  xd[4] = xd[4] - g;
  xd[7] = 0.5 * (-q[1] * wx - q[2] * wy - q[3] * wz);
  xd[8] = 0.5 * (q[0] * wx + q[2] * wz - q[3] * wy);
  xd[9] = 0.5 * (q[0] * wy - q[1] * wz + q[3] * wx);
  xd[10] = 0.5 * (q[0] * wz + q[1] * wy - q[2] * wx);
  xd[11] = (-(Jz - Jy) * wy * wz) / Jx;
  xd[12] = (l * u[2] - (Jx - Jz) * wz * wx) / Jy;
  xd[13] = (-l * u[1] - (Jy - Jx) * wx * wy) / Jz;
}

int model_nx(int model) {
  return model == MODEL_QUAD12 ? 12 : (model == MODEL_QUAT13 ? 13 : (model == MODEL_MARS14 ? 14 : 7));
}
int model_nu(int model) { return (model == MODEL_MARS7 || model == MODEL_MARS14) ? 3 : 4; }

template <class S>
void f_eval(int model, const double* prm, const S* x, const S* u, S* xd) {
  if (model == MODEL_QUAD12) quad_f<S>(prm, x, u, xd);
  else if (model == MODEL_QUAT13) quat_f<S>(prm, x, u, xd);
  else if (model == MODEL_MARS14) mars6_f<S>(prm, x, u, xd);
  else mars_f<S>(prm, x, u, xd);
}

// Classical RK4 step of length h (Eq. (1b)).
template <class S>
void rk4(int model, const double* prm, double h, const S* x, const S* u, S* xn) {
  const int nx = model_nx(model);
  S k1[16], k2[16], k3[16], k4[16], t[16];
  f_eval<S>(model, prm, x, u, k1);
  for (int j = 0; j < nx; ++j) t[j] = x[j] + (0.5 * h) * k1[j];
  f_eval<S>(model, prm, t, u, k2);
  for (int j = 0; j < nx; ++j) t[j] = x[j] + (0.5 * h) * k2[j];
  f_eval<S>(model, prm, t, u, k3);
  for (int j = 0; j < nx; ++j) t[j] = x[j] + h * k3[j];
  f_eval<S>(model, prm, t, u, k4);
  for (int j = 0; j < nx; ++j) xn[j] = x[j] + (h / 6.0) * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
}

// Hand-derived Jacobians f_x (nx*nx row-major) and f_u (nx*nu).
void quad_jac(const double* prm, const double* x, const double* u, double* fx, double* fu) {
  const int nx = 12, nu = 4;
  const double m = prm[0], Jx = prm[1], Jy = prm[2], Jz = prm[3];
  const double l = prm[4], km = prm[5], cd = prm[6];
  std::fill(fx, fx + nx * nx, 0.0);
  std::fill(fu, fu + nx * nu, 0.0);
  const double ph = x[6], th = x[7], ps = x[8];
  const double sphi = std::sin(ph), cphi = std::cos(ph);
  const double sth = std::sin(th), cth = std::cos(th);
  const double sps = std::sin(ps), cps = std::cos(ps);
  const double F = u[0] + u[1] + u[2] + u[3];
  const double a[3] = {cphi * sth * cps + sphi * sps, cphi * sth * sps - sphi * cps, cphi * cth};
  const double da_dphi[3] = {-sphi * sth * cps + cphi * sps, -sphi * sth * sps - cphi * cps, -sphi * cth};
  const double da_dth[3] = {cphi * cth * cps, cphi * cth * sps, -cphi * sth};
  const double da_dps[3] = {-cphi * sth * sps + sphi * cps, cphi * sth * cps + sphi * sps, 0.0};
  for (int k = 0; k < 3; ++k) fx[k * nx + 3 + k] = 1.0;              // p' = v
  for (int k = 0; k < 3; ++k) {
    fx[(3 + k) * nx + 3 + k] = -cd / m;
    fx[(3 + k) * nx + 6] = da_dphi[k] * F / m;
    fx[(3 + k) * nx + 7] = da_dth[k] * F / m;
    fx[(3 + k) * nx + 8] = da_dps[k] * F / m;
    for (int j = 0; j < 4; ++j) fu[(3 + k) * nu + j] = a[k] / m;
  }
  const double wx = x[9], wy = x[10], wz = x[11];
  const double tth = sth / cth, sec2 = 1.0 / (cth * cth);
  // phi' = wx + tan(th) (sphi wy + cphi wz)
  fx[6 * nx + 6] = tth * (cphi * wy - sphi * wz);
  fx[6 * nx + 7] = sec2 * (sphi * wy + cphi * wz);
  fx[6 * nx + 9] = 1.0;
  fx[6 * nx + 10] = sphi * tth;
  fx[6 * nx + 11] = cphi * tth;
  // th' = cphi wy - sphi wz
  fx[7 * nx + 6] = -sphi * wy - cphi * wz;
  fx[7 * nx + 10] = cphi;
  fx[7 * nx + 11] = -sphi;
  // psi' = (sphi wy + cphi wz) / cth
  fx[8 * nx + 6] = (cphi * wy - sphi * wz) / cth;
  fx[8 * nx + 7] = (sphi * wy + cphi * wz) * sth / (cth * cth);
  fx[8 * nx + 10] = sphi / cth;
  fx[8 * nx + 11] = cphi / cth;
  // omega' = J^-1 (tau - omega x J omega)
  fx[9 * nx + 10] = -(Jz - Jy) * wz / Jx;
  fx[9 * nx + 11] = -(Jz - Jy) * wy / Jx;
  fx[10 * nx + 9] = -(Jx - Jz) * wz / Jy;
  fx[10 * nx + 11] = -(Jx - Jz) * wx / Jy;
  fx[11 * nx + 9] = -(Jy - Jx) * wy / Jz;
  fx[11 * nx + 10] = -(Jy - Jx) * wx / Jz;
  fu[9 * nu + 1] = l / Jx;  fu[9 * nu + 3] = -l / Jx;
  fu[10 * nu + 0] = -l / Jy; fu[10 * nu + 2] = l / Jy;
  fu[11 * nu + 0] = km / Jz; fu[11 * nu + 1] = -km / Jz;
  fu[11 * nu + 2] = km / Jz; fu[11 * nu + 3] = -km / Jz;
}

void mars_jac(const double* prm, const double* x, const double* u, double* fx, double* fu) {
  const int nx = 7, nu = 3;
  const double alpha = prm[1];
  std::fill(fx, fx + nx * nx, 0.0);
  std::fill(fu, fu + nx * nu, 0.0);
  const double m = x[6];
  for (int k = 0; k < 3; ++k) {
    fx[k * nx + 3 + k] = 1.0;
    fx[(3 + k) * nx + 6] = -u[k] / (m * m);
    fu[(3 + k) * nu + k] = 1.0 / m;
  }
  const double Tn = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (Tn > 0.0)
    for (int k = 0; k < 3; ++k) fu[6 * nu + k] = -alpha * u[k] / Tn;
}

void quat_jac(const double* prm, const double* x, const double* u, double* fx, double* fu) {
  const int nx = 13, nu = 4;
  const double m = prm[0], Jx = prm[1], Jy = prm[2], Jz = prm[3], cd = prm[6];
  std::fill(fx, fx + nx * nx, 0.0);
  std::fill(fu, fu + nx * nu, 0.0);
  const double qw = x[6], qx = x[7], qy = x[8], qz = x[9];
  const double wx = x[10], wy = x[11], wz = x[12];
  const double T = u[0];
  const double a[3] = {2.0 * (qx * qz + qw * qy), 2.0 * (qy * qz - qw * qx), qw * qw - qx * qx - qy * qy + qz * qz};
  // d a_k / d (qw, qx, qy, qz)
  const double da[3][4] = {{2.0 * qy, 2.0 * qz, 2.0 * qw, 2.0 * qx},
                           {-2.0 * qx, -2.0 * qw, 2.0 * qz, 2.0 * qy},
                           {2.0 * qw, -2.0 * qx, -2.0 * qy, 2.0 * qz}};
  for (int k = 0; k < 3; ++k) fx[k * nx + 3 + k] = 1.0;              // r' = v
  for (int k = 0; k < 3; ++k) {
    fx[(3 + k) * nx + 3 + k] = -cd / m;
    for (int j = 0; j < 4; ++j) fx[(3 + k) * nx + 6 + j] = da[k][j] * T / m;
    fu[(3 + k) * nu + 0] = a[k] / m;
  }
  // q' = 1/2 Omega(omega) q: rows qw', qx', qy', qz' over (qw, qx, qy, qz)
  const double Om[4][4] = {{0.0, -wx, -wy, -wz}, {wx, 0.0, wz, -wy}, {wy, -wz, 0.0, wx}, {wz, wy, -wx, 0.0}};
  // ... and over (wx, wy, wz)
  const double Qm[4][3] = {{-qx, -qy, -qz}, {qw, -qz, qy}, {qz, qw, -qx}, {-qy, qx, qw}};
  for (int r = 0; r < 4; ++r) {
    for (int c = 0; c < 4; ++c) fx[(6 + r) * nx + 6 + c] = 0.5 * Om[r][c];
    for (int c = 0; c < 3; ++c) fx[(6 + r) * nx + 10 + c] = 0.5 * Qm[r][c];
  }
  // omega' = J^-1 (tau - omega x J omega)
  fx[10 * nx + 11] = -(Jz - Jy) * wz / Jx;
  fx[10 * nx + 12] = -(Jz - Jy) * wy / Jx;
  fx[11 * nx + 10] = -(Jx - Jz) * wz / Jy;
  fx[11 * nx + 12] = -(Jx - Jz) * wx / Jy;
  fx[12 * nx + 10] = -(Jy - Jx) * wy / Jz;
  fx[12 * nx + 11] = -(Jy - Jx) * wx / Jz;
  fu[10 * nu + 1] = 1.0 / Jx;
  fu[11 * nu + 2] = 1.0 / Jy;
  fu[12 * nu + 3] = 1.0 / Jz;
}

void mars6_jac(const double* prm, const double* x, const double* u, double* fx, double* fu) {
  const int nx = 14, nu = 3;
  const double alpha = prm[0], Jx = prm[2], Jy = prm[3], Jz = prm[4], l = prm[5];
  std::fill(fx, fx + nx * nx, 0.0);
  std::fill(fu, fu + nx * nu, 0.0);
  const double m = x[0];
  const double qw = x[7], qa = x[8], qb = x[9], qc = x[10];
  const double wx = x[11], wy = x[12], wz = x[13];
  double C[3][3];
  quat_rot<double>(&x[7], C);
  // d C[k][j] / d (qw, qx, qy, qz)
  const double dC[3][3][4] = {
      {{2 * qw, 2 * qa, -2 * qb, -2 * qc}, {-2 * qc, 2 * qb, 2 * qa, -2 * qw}, {2 * qb, 2 * qc, 2 * qw, 2 * qa}},
      {{2 * qc, 2 * qb, 2 * qa, 2 * qw}, {2 * qw, -2 * qa, 2 * qb, -2 * qc}, {-2 * qa, -2 * qw, 2 * qc, 2 * qb}},
      {{-2 * qb, 2 * qc, -2 * qw, 2 * qa}, {2 * qa, 2 * qw, 2 * qc, 2 * qb}, {2 * qw, -2 * qa, -2 * qb, 2 * qc}}};
  const double Tn = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  if (Tn > 0.0)
    for (int j = 0; j < 3; ++j) fu[0 * nu + j] = -alpha * u[j] / Tn;
  for (int k = 0; k < 3; ++k) fx[(1 + k) * nx + 4 + k] = 1.0;                 // r' = v
  for (int k = 0; k < 3; ++k) {
    const double CT = C[k][0] * u[0] + C[k][1] * u[1] + C[k][2] * u[2];
    fx[(4 + k) * nx + 0] = -CT / (m * m);
    for (int a = 0; a < 4; ++a) {
      double acc = 0.0;
      for (int j = 0; j < 3; ++j) acc += dC[k][j][a] * u[j];
      fx[(4 + k) * nx + 7 + a] = acc / m;
    }
    for (int j = 0; j < 3; ++j) fu[(4 + k) * nu + j] = C[k][j] / m;
  }
  const double Om[4][4] = {{0.0, -wx, -wy, -wz}, {wx, 0.0, wz, -wy}, {wy, -wz, 0.0, wx}, {wz, wy, -wx, 0.0}};
  const double Qm[4][3] = {{-qa, -qb, -qc}, {qw, -qc, qb}, {qc, qw, -qa}, {-qb, qa, qw}};
  for (int r = 0; r < 4; ++r) {
    for (int c = 0; c < 4; ++c) fx[(7 + r) * nx + 7 + c] = 0.5 * Om[r][c];
    for (int c = 0; c < 3; ++c) fx[(7 + r) * nx + 11 + c] = 0.5 * Qm[r][c];
  }
  fx[11 * nx + 12] = -(Jz - Jy) * wz / Jx;
  fx[11 * nx + 13] = -(Jz - Jy) * wy / Jx;
  fx[12 * nx + 11] = -(Jx - Jz) * wz / Jy;
  fx[12 * nx + 13] = -(Jx - Jz) * wx / Jy;
  fx[13 * nx + 11] = -(Jy - Jx) * wy / Jz;
  fx[13 * nx + 12] = -(Jy - Jx) * wx / Jz;
  fu[12 * nu + 2] = l / Jy;
  fu[13 * nu + 1] = -l / Jz;
}

void f_jac(int model, const double* prm, const double* x, const double* u, double* fx, double* fu) {
  if (model == MODEL_QUAD12) quad_jac(prm, x, u, fx, fu);
  else if (model == MODEL_QUAT13) quat_jac(prm, x, u, fx, fu);
  else if (model == MODEL_MARS14) mars6_jac(prm, x, u, fx, fu);
  else mars_jac(prm, x, u, fx, fu);
}

// RK4 step and its sensitivity Phi = d x_next / d(x, u)  (nx x (nx+nu)),
// by differentiating each stage: K_s = f_x(x_s) X_s + [0, f_u(x_s)] with
// X_1 = [I 0], X_2 = X_1 + h/2 K_1, X_3 = X_1 + h/2 K_2, X_4 = X_1 + h K_3,
// Phi = [I 0] + h/6 (K_1 + 2 K_2 + 2 K_3 + K_4).
void rk4_variational(int model, const double* prm, double h, const double* x, const double* u,
                     double* xn, double* A, double* B) {
  const int nx = model_nx(model), nu = model_nu(model), n = nx + nu;
  std::vector<double> X0(nx * n, 0.0), Xs(nx * n), K[4], Phi(nx * n);
  for (int j = 0; j < nx; ++j) X0[j * n + j] = 1.0;
  double xs[16], k[4][16], fx[256], fu[128];
  const double cstage[4] = {0.0, 0.5 * h, 0.5 * h, h};
  for (int s = 0; s < 4; ++s) {
    K[s].assign(nx * n, 0.0);
    // stage point and its sensitivity
    for (int j = 0; j < nx; ++j) xs[j] = (s == 0) ? x[j] : x[j] + cstage[s] * k[s - 1][j];
    for (int e = 0; e < nx * n; ++e) Xs[e] = (s == 0) ? X0[e] : X0[e] + cstage[s] * K[s - 1][e];
    f_eval<double>(model, prm, xs, u, k[s]);
    f_jac(model, prm, xs, u, fx, fu);
    for (int r = 0; r < nx; ++r)
      for (int c = 0; c < n; ++c) {
        double acc = 0.0;
        for (int q = 0; q < nx; ++q) acc += fx[r * nx + q] * Xs[q * n + c];
        if (c >= nx) acc += fu[r * nu + (c - nx)];
        K[s][r * n + c] = acc;
      }
  }
  for (int j = 0; j < nx; ++j) xn[j] = x[j] + (h / 6.0) * (k[0][j] + 2.0 * k[1][j] + 2.0 * k[2][j] + k[3][j]);
  for (int e = 0; e < nx * n; ++e)
    Phi[e] = X0[e] + (h / 6.0) * (K[0][e] + 2.0 * K[1][e] + 2.0 * K[2][e] + K[3][e]);
  for (int r = 0; r < nx; ++r) {
    for (int c = 0; c < nx; ++c) A[r * nx + c] = Phi[r * n + c];
    for (int c = 0; c < nu; ++c) B[r * nu + c] = Phi[r * n + nx + c];
  }
}

// ============================================================= projections
// Half-space {s : s >= b} for a scalar mirror s = n^T y (unit n): clamp from below.
double proj_half(double s, double b) { return s < b ? b : s; }

// Ball {y : |y| <= R}: vector scaling (Sec. II, "norm constraints ... vector scaling").
void proj_ball(const double* y, int dim, double R, double* out) {
  double nn = 0.0;
  for (int k = 0; k < dim; ++k) nn += y[k] * y[k];
  nn = std::sqrt(nn);
  double sc = (nn > R) ? R / nn : 1.0;
  for (int k = 0; k < dim; ++k) out[k] = y[k] * sc;
}

// Second-order cone {(t, y) : |y| <= tau t} with t = first component, y = the
// other two.  Standard three-case projection onto a Lorentz cone of
// half-angle atan(tau) (Parikh & Boyd, Proximal Algorithms, Sec. 6.3.2):
//   inside -> unchanged; inside the polar cone (tau |y| <= -t) -> 0;
//   else onto the boundary ray: c = t cos(a) + |y| sin(a), (t,y) -> c (cos a, sin a y/|y|).
void proj_cone(const double* v, double tau, double* out) {
  const double t = v[0], s = std::sqrt(v[1] * v[1] + v[2] * v[2]);
  if (s <= tau * t) { out[0] = v[0]; out[1] = v[1]; out[2] = v[2]; return; }
  if (tau * s <= -t) { out[0] = out[1] = out[2] = 0.0; return; }
  const double ca = 1.0 / std::sqrt(1.0 + tau * tau), sa = tau * ca;
  const double c = t * ca + s * sa;
  out[0] = c * ca;
  out[1] = c * sa * v[1] / s;
  out[2] = c * sa * v[2] / s;
}

void proj_block(int kind, int dim, double p0, const double* y, double* out) {
  if (kind == BLK_HALF) out[0] = proj_half(y[0], p0);
  else if (kind == BLK_BALL) proj_ball(y, dim, p0, out);
  else if (kind == BLK_CONE) proj_cone(y, p0, out);
  else for (int k = 0; k < dim; ++k) out[k] = y[k];
}

int blk_dim(int kind) { return kind == BLK_HALF ? 1 : (kind == BLK_NONE ? 0 : 3); }

// ============================================================= the QP of Eq. (2)
struct Block {
  int kind = BLK_NONE;
  std::vector<double> G;  // 3 x n row-major (rows beyond dim unused)
  double p0 = 0.0;
};

struct QPNode {
  std::vector<double> A, B, d;      // dynamics to node i+1 (i < N)
  std::vector<double> Q, R, M;      // cost Hessian blocks (full)
  std::vector<double> q, r;         // cost gradient
  std::vector<double> xlo, xhi, ulo, uhi;  // boxes (already intersected with the trust region)
  std::vector<Block> blk;           // mirror blocks
};

struct QP {
  int N = 0, nx = 0, nu = 0, maxblk = 0;
  std::vector<QPNode> node;         // N+1 nodes
  std::vector<double> xinit, xtarget;
  std::vector<unsigned char> tmask;
  double rho_eq = 1, rho_dyn = 1, rho_geo = 1;
};

// ADMM variables, absolute coordinates (the paper's form, Eq. (3)).
struct State {
  int N, nx, nu, mb;
  std::vector<double> x, u, z, lam, mu, xh, uh, nux, nuu, s, nus;
  void alloc(int N_, int nx_, int nu_, int mb_) {
    N = N_; nx = nx_; nu = nu_; mb = mb_;
    x.assign((N + 1) * nx, 0); u.assign(N * nu, 0); z.assign((N + 1) * nx, 0);
    lam.assign((N + 1) * nx, 0); mu.assign((N + 1) * nx, 0); xh.assign((N + 1) * nx, 0);
    uh.assign(N * nu, 0); nux.assign((N + 1) * nx, 0); nuu.assign(N * nu, 0);
    s.assign((N + 1) * mb * 3, 0); nus.assign((N + 1) * mb * 3, 0);
  }
  // Flat export order: x, u, z, lam, mu, xh, uh, nux, nuu, s, nus.
  size_t size() const { return x.size() + u.size() + z.size() + lam.size() + mu.size() + xh.size() + uh.size() + nux.size() + nuu.size() + s.size() + nus.size(); }
  void to_flat(double* o) const {
    for (const std::vector<double>* v : {&x, &u, &z, &lam, &mu, &xh, &uh, &nux, &nuu, &s, &nus}) {
      std::memcpy(o, v->data(), v->size() * sizeof(double)); o += v->size();
    }
  }
  void from_flat(const double* o) {
    for (std::vector<double>* v : {&x, &u, &z, &lam, &mu, &xh, &uh, &nux, &nuu, &s, &nus}) {
      std::memcpy(v->data(), o, v->size() * sizeof(double)); o += v->size();
    }
  }
};

size_t state_size(int N, int nx, int nu, int mb) {
  return (size_t)6 * (N + 1) * nx + (size_t)3 * N * nu + (size_t)2 * (N + 1) * mb * 3;
}

// xi = [x_i; u_i] (u absent at node N).
void node_xi(const State& st, int i, double* xi) {
  for (int j = 0; j < st.nx; ++j) xi[j] = st.x[i * st.nx + j];
  if (i < st.N) for (int j = 0; j < st.nu; ++j) xi[st.nx + j] = st.u[i * st.nu + j];
}

void block_apply(const Block& b, int n, const double* xi, double* out) {
  const int dim = blk_dim(b.kind);
  for (int r = 0; r < dim; ++r) {
    double acc = 0.0;
    for (int c = 0; c < n; ++c) acc += b.G[r * n + c] * xi[c];
    out[r] = acc;
  }
}

// Unpivoted Cholesky H = L L^T in place (lower triangle).  Returns false on a
// non-positive pivot.  H_i is SPD by the rho terms (Sec. III-B, Step 1).
bool cholesky(std::vector<double>& H, int n) {
  for (int j = 0; j < n; ++j) {
    double s = H[j * n + j];
    for (int k = 0; k < j; ++k) s -= H[j * n + k] * H[j * n + k];
    if (!(s > 0.0)) return false;
    const double Ljj = std::sqrt(s);
    H[j * n + j] = Ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = H[i * n + j];
      for (int k = 0; k < j; ++k) t -= H[i * n + k] * H[j * n + k];
      H[i * n + j] = t / Ljj;
    }
  }
  return true;
}

// Forward then backward substitution with the cached factor.
void chol_solve(const std::vector<double>& L, int n, const double* g, double* xi) {
  double y[32];
  for (int i = 0; i < n; ++i) {
    double t = g[i];
    for (int k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
    y[i] = t / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * xi[k];
    xi[i] = t / L[i * n + i];
  }
}

// H_i of Eq. (4), extended by rho_geo G_j^T G_j for every mirror block.
std::vector<double> build_H(const QP& qp, int i) {
  const int nx = qp.nx, nu = qp.nu, N = qp.N;
  const int n = (i < N) ? nx + nu : nx;
  const QPNode& nd = qp.node[i];
  std::vector<double> H(n * n, 0.0);
  for (int r = 0; r < nx; ++r)
    for (int c = 0; c < nx; ++c) H[r * n + c] = nd.Q[r * nx + c];
  for (int r = 0; r < nx; ++r) H[r * n + r] += qp.rho_geo + (i > 0 ? qp.rho_eq : 0.0);
  if (i < N) {
    for (int r = 0; r < nx; ++r)
      for (int c = 0; c < nx; ++c) {
        double acc = 0.0;
        for (int k = 0; k < nx; ++k) acc += nd.A[k * nx + r] * nd.A[k * nx + c];
        H[r * n + c] += qp.rho_dyn * acc;
      }
    for (int r = 0; r < nx; ++r)
      for (int c = 0; c < nu; ++c) {
        double acc = 0.0;
        for (int k = 0; k < nx; ++k) acc += nd.A[k * nx + r] * nd.B[k * nu + c];
        const double h12 = nd.M[r * nu + c] + qp.rho_dyn * acc;
        H[r * n + nx + c] = h12;
        H[(nx + c) * n + r] = h12;       // H_21 = H_12^T
      }
    for (int r = 0; r < nu; ++r)
      for (int c = 0; c < nu; ++c) {
        double acc = 0.0;
        for (int k = 0; k < nx; ++k) acc += nd.B[k * nu + r] * nd.B[k * nu + c];
        H[(nx + r) * n + nx + c] = nd.R[r * nu + c] + qp.rho_dyn * acc + (r == c ? qp.rho_geo : 0.0);
      }
  }
  for (const Block& b : nd.blk) {
    const int dim = blk_dim(b.kind);
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double acc = 0.0;
        for (int k = 0; k < dim; ++k) acc += b.G[k * n + r] * b.G[k * n + c];
        H[r * n + c] += qp.rho_geo * acc;
      }
  }
  return H;
}

void project_xhat(const QP& qp, int i, const double* v, double* out) {
  const int nx = qp.nx;
  const QPNode& nd = qp.node[i];
  for (int j = 0; j < nx; ++j) {
    if (i == 0) out[j] = qp.xinit[j];                              // X_0 = {x_init}
    else if (i == qp.N && qp.tmask[j]) out[j] = qp.xtarget[j];     // S x_N = x_target
    else out[j] = std::min(std::max(v[j], nd.xlo[j]), nd.xhi[j]); // clamp, Eq. (7)
  }
}

void init_state(const QP& qp, const double* xbar, const double* ubar, State& st) {
  const int N = qp.N, nx = qp.nx, nu = qp.nu, n1 = nx + nu;
  st.alloc(N, nx, nu, qp.maxblk);
  for (int e = 0; e < (N + 1) * nx; ++e) { st.x[e] = st.xh[e] = xbar[e]; }
  for (int i = 1; i <= N; ++i)
    for (int j = 0; j < nx; ++j) st.z[i * nx + j] = xbar[i * nx + j];
  for (int e = 0; e < N * nu; ++e) { st.u[e] = st.uh[e] = ubar[e]; }
  double xi[32], y[3];
  for (int i = 0; i <= N; ++i) {
    const int n = (i < N) ? n1 : nx;
    node_xi(st, i, xi);
    for (int b = 0; b < qp.maxblk; ++b) {
      const Block& B = qp.node[i].blk[b];
      if (B.kind == BLK_NONE) continue;
      block_apply(B, n, xi, y);
      proj_block(B.kind, blk_dim(B.kind), B.p0, y, &st.s[(i * qp.maxblk + b) * 3]);
    }
  }
}

// Re-project every mirror from the current (x-hat, u-hat) with this QP's G_j.
void reseed_mirrors(const QP& qp, State& st) {
  const int N = qp.N, nx = qp.nx, nu = qp.nu;
  double xi[32], y[3];
  for (int i = 0; i <= N; ++i) {
    const int n = (i < N) ? nx + nu : nx;
    for (int j = 0; j < nx; ++j) xi[j] = st.xh[i * nx + j];
    if (i < N) for (int j = 0; j < nu; ++j) xi[nx + j] = st.uh[i * nu + j];
    for (int b = 0; b < qp.maxblk; ++b) {
      const Block& B = qp.node[i].blk[b];
      double* sp = &st.s[(i * qp.maxblk + b) * 3];
      if (B.kind == BLK_NONE) { sp[0] = sp[1] = sp[2] = 0.0; continue; }
      block_apply(B, n, xi, y);
      proj_block(B.kind, blk_dim(B.kind), B.p0, y, sp);
    }
  }
}

struct AdmmStats { double primal = 0, dual = 0; int ok = 1; };

// Work space of one ADMM call: the cached factors (H_i is constant within an
// SCP iteration) and what the last iteration's residuals need.
struct AdmmWork {
  std::vector<std::vector<double>> L;
  std::vector<double> dd, zold, xhold, uhold, sold;
};

bool admm_prepare(const QP& qp, AdmmWork& wk) {
  const int N = qp.N, nx = qp.nx, nu = qp.nu, n1 = nx + nu;
  wk.L.assign(N + 1, std::vector<double>());
  for (int i = 0; i <= N; ++i) {
    wk.L[i] = build_H(qp, i);
    if (!cholesky(wk.L[i], (i < N) ? n1 : nx)) return false;
  }
  wk.dd.assign(N * nx, 0.0);
  return true;
}

// First part of one ADMM iteration: Step 1, the linearised propagation,
// Step 2 and Step 3.
void admm_first_part(const QP& qp, State& st, AdmmWork& wk, bool last) {
  const int N = qp.N, nx = qp.nx, nu = qp.nu, n1 = nx + nu, mb = qp.maxblk;
  const double re = qp.rho_eq, rd = qp.rho_dyn, rg = qp.rho_geo;
  const std::vector<std::vector<double>>& L = wk.L;
  std::vector<double>& dd = wk.dd;
  double g[32], xi[32], y[3], w[16];
  (void)re;
    // ---- Step 1: per-node KKT solve H_i xi_i = g_i
    for (int i = 0; i <= N; ++i) {
      const QPNode& nd = qp.node[i];
      const int n = (i < N) ? n1 : nx;
      for (int j = 0; j < nx; ++j) {
        double v = -nd.q[j] + rg * st.xh[i * nx + j] - st.nux[i * nx + j];
        if (i > 0) v += re * st.z[i * nx + j] - st.lam[i * nx + j];
        g[j] = v;
      }
      if (i < N) {
        // w_i = mu_{i+1} + rho_dyn (z_{i+1} - d_i): the dynamic-coupling pull from node i+1
        for (int k = 0; k < nx; ++k) w[k] = st.mu[(i + 1) * nx + k] + rd * (st.z[(i + 1) * nx + k] - nd.d[k]);
        for (int j = 0; j < nx; ++j) {
          double acc = 0.0;
          for (int k = 0; k < nx; ++k) acc += nd.A[k * nx + j] * w[k];
          g[j] += acc;
        }
        for (int j = 0; j < nu; ++j) {
          double acc = 0.0;
          for (int k = 0; k < nx; ++k) acc += nd.B[k * nu + j] * w[k];
          g[nx + j] = -nd.r[j] + acc + rg * st.uh[i * nu + j] - st.nuu[i * nu + j];
        }
      }
      for (int b = 0; b < mb; ++b) {
        const Block& B = nd.blk[b];
        if (B.kind == BLK_NONE) continue;
        const int dim = blk_dim(B.kind);
        for (int c = 0; c < n; ++c) {
          double acc = 0.0;
          for (int k = 0; k < dim; ++k)
            acc += B.G[k * n + c] * (rg * st.s[(i * mb + b) * 3 + k] - st.nus[(i * mb + b) * 3 + k]);
          g[c] += acc;
        }
      }
      chol_solve(L[i], n, g, xi);
      for (int j = 0; j < nx; ++j) st.x[i * nx + j] = xi[j];
      if (i < N) for (int j = 0; j < nu; ++j) st.u[i * nu + j] = xi[nx + j];
    }
    // linearised propagation d_dyn,i = A_i x_i + B_i u_i + d_i
    for (int i = 0; i < N; ++i) {
      const QPNode& nd = qp.node[i];
      for (int r = 0; r < nx; ++r) {
        double acc = nd.d[r];
        for (int c = 0; c < nx; ++c) acc += nd.A[r * nx + c] * st.x[i * nx + c];
        for (int c = 0; c < nu; ++c) acc += nd.B[r * nu + c] * st.u[i * nu + c];
        dd[i * nx + r] = acc;
      }
    }
    if (last) { wk.zold = st.z; wk.xhold = st.xh; wk.uhold = st.uh; wk.sold = st.s; }
    // ---- Step 2: dynamic consensus, Eq. (5)
    for (int i = 1; i <= N; ++i)
      for (int j = 0; j < nx; ++j)
        st.z[i * nx + j] = (re * st.x[i * nx + j] + st.lam[i * nx + j] + rd * dd[(i - 1) * nx + j] - st.mu[i * nx + j]) / (re + rd);
    // ---- Step 3: geometric projections (Eq. (6)-(7) and the mirror sets)
    for (int i = 0; i <= N; ++i) {
      double v[16], o[16];
      for (int j = 0; j < nx; ++j) v[j] = st.x[i * nx + j] + st.nux[i * nx + j] / rg;
      project_xhat(qp, i, v, o);
      for (int j = 0; j < nx; ++j) st.xh[i * nx + j] = o[j];
      if (i < N)
        for (int j = 0; j < nu; ++j) {
          const double t = st.u[i * nu + j] + st.nuu[i * nu + j] / rg;
          st.uh[i * nu + j] = std::min(std::max(t, qp.node[i].ulo[j]), qp.node[i].uhi[j]);
        }
      const int n = (i < N) ? n1 : nx;
      node_xi(st, i, xi);
      for (int b = 0; b < mb; ++b) {
        const Block& B = qp.node[i].blk[b];
        if (B.kind == BLK_NONE) continue;
        const int dim = blk_dim(B.kind);
        block_apply(B, n, xi, y);
        double t[3];
        for (int k = 0; k < dim; ++k) t[k] = y[k] + st.nus[(i * mb + b) * 3 + k] / rg;
        proj_block(B.kind, dim, B.p0, t, &st.s[(i * mb + b) * 3]);
      }
    }
}

// Second part: Step 4 (dual ascent) and, on the last iteration, the residuals.
void admm_second_part(const QP& qp, State& st, AdmmWork& wk, bool last, AdmmStats& out) {
  const int N = qp.N, nx = qp.nx, nu = qp.nu, n1 = nx + nu, mb = qp.maxblk;
  const double re = qp.rho_eq, rd = qp.rho_dyn, rg = qp.rho_geo;
  std::vector<double>& dd = wk.dd;
  double xi[32], y[3], w[16];
    // ---- Step 4: dual ascent, Eq. (8) and its analogues
    for (int i = 1; i <= N; ++i)
      for (int j = 0; j < nx; ++j) {
        st.lam[i * nx + j] += re * (st.x[i * nx + j] - st.z[i * nx + j]);
        st.mu[i * nx + j] += rd * (st.z[i * nx + j] - dd[(i - 1) * nx + j]);
      }
    for (int e = 0; e < (N + 1) * nx; ++e) st.nux[e] += rg * (st.x[e] - st.xh[e]);
    for (int e = 0; e < N * nu; ++e) st.nuu[e] += rg * (st.u[e] - st.uh[e]);
    for (int i = 0; i <= N; ++i) {
      const int n = (i < N) ? n1 : nx;
      node_xi(st, i, xi);
      for (int b = 0; b < mb; ++b) {
        const Block& B = qp.node[i].blk[b];
        if (B.kind == BLK_NONE) continue;
        block_apply(B, n, xi, y);
        for (int k = 0; k < blk_dim(B.kind); ++k)
          st.nus[(i * mb + b) * 3 + k] += rg * (y[k] - st.s[(i * mb + b) * 3 + k]);
      }
    }
    if (last) {
      // primal residual: all consensus constraints at the final iterate
      double rp = 0.0, rdl = 0.0;
      for (int i = 1; i <= N; ++i)
        for (int j = 0; j < nx; ++j) {
          const double a = st.x[i * nx + j] - st.z[i * nx + j];
          const double b = st.z[i * nx + j] - dd[(i - 1) * nx + j];
          rp += a * a + b * b;
        }
      for (int e = 0; e < (N + 1) * nx; ++e) { const double a = st.x[e] - st.xh[e]; rp += a * a; }
      for (int e = 0; e < N * nu; ++e) { const double a = st.u[e] - st.uh[e]; rp += a * a; }
      for (int i = 0; i <= N; ++i) {
        const int n = (i < N) ? n1 : nx;
        node_xi(st, i, xi);
        for (int b = 0; b < mb; ++b) {
          const Block& B = qp.node[i].blk[b];
          if (B.kind == BLK_NONE) continue;
          block_apply(B, n, xi, y);
          for (int k = 0; k < blk_dim(B.kind); ++k) { const double a = y[k] - st.s[(i * mb + b) * 3 + k]; rp += a * a; }
        }
      }
      // dual residual of the last step: rho P^T Q (v_new - v_old) for the
      // second block v = (z, x-hat, u-hat, s), per node in xi coordinates
      for (int i = 0; i <= N; ++i) {
        const int n = (i < N) ? n1 : nx;
        const QPNode& nd = qp.node[i];
        double sv[32];
        for (int c = 0; c < n; ++c) sv[c] = 0.0;
        for (int j = 0; j < nx; ++j) {
          sv[j] += rg * (st.xh[i * nx + j] - wk.xhold[i * nx + j]);
          if (i > 0) sv[j] += re * (st.z[i * nx + j] - wk.zold[i * nx + j]);
        }
        if (i < N) {
          for (int k = 0; k < nx; ++k) w[k] = rd * (st.z[(i + 1) * nx + k] - wk.zold[(i + 1) * nx + k]);
          for (int j = 0; j < nx; ++j) for (int k = 0; k < nx; ++k) sv[j] += nd.A[k * nx + j] * w[k];
          for (int j = 0; j < nu; ++j) {
            for (int k = 0; k < nx; ++k) sv[nx + j] += nd.B[k * nu + j] * w[k];
            sv[nx + j] += rg * (st.uh[i * nu + j] - wk.uhold[i * nu + j]);
          }
        }
        for (int b = 0; b < mb; ++b) {
          const Block& B = nd.blk[b];
          if (B.kind == BLK_NONE) continue;
          for (int c = 0; c < n; ++c)
            for (int k = 0; k < blk_dim(B.kind); ++k)
              sv[c] += rg * B.G[k * n + c] * (st.s[(i * mb + b) * 3 + k] - wk.sold[(i * mb + b) * 3 + k]);
        }
        for (int c = 0; c < n; ++c) rdl += sv[c] * sv[c];
      }
      out.primal = std::sqrt(rp);
      out.dual = std::sqrt(rdl);
    }
}

// `iters` ADMM iterations (Sec. III-B, Steps 1-4) on the QP, in place.
AdmmStats admm_run(const QP& qp, State& st, int iters) {
  AdmmStats out;
  AdmmWork wk;
  if (!admm_prepare(qp, wk)) { out.ok = 0; return out; }
  for (int it = 0; it < iters; ++it) {
    const bool last = (it == iters - 1);
    admm_first_part(qp, st, wk, last);
    admm_second_part(qp, st, wk, last, out);
  }
  return out;
}

// ============================================================= problem -> QP (Sec. III-A)
}  // namespace

extern "C" {

// The oracle's own view of a problem batch (arrays per instance, row-major).
struct OrcProblem {
  int model, nx, nu, batch;
  const int* N;
  const long long* xoff;
  const long long* uoff;
  const double* dt;
  const double* params;   // [B][8]
  const double* Qd; const double* xref; const double* Rd; const double* uref;
  const double* QNd; const double* qN;
  const double* xlo; const double* xhi; const double* ulo; const double* uhi;
  const double* xinit; const double* xtarget; const unsigned char* tmask;
  int max_obs; const int* nobs; const double* obs_c; const double* obs_r;
  const double* sets;     // [B][8]: thrust_min, thrust_max, tan(glide), then model-specific
  double rho_eq, rho_dyn, rho_geo, rho_final;
  int scp_iters, admm_iters, stop;
  double tr_init, tr_min, tr_max, w_d, defect_tol, step_tol, vc_weight;
  int group;              // scenarios per group (1: independent instances)
};

}  // extern "C"

namespace {

int problem_maxblk(const OrcProblem& P) {
  return P.model == MODEL_MARS7 ? 3 : (P.model == MODEL_MARS14 ? 6 : P.max_obs);
}

// Build the QP of Eq. (2) at nominal (xbar, ubar) for instance b: exact
// quadratic cost expansion, trust-region l_inf box of radius `radius`
// intersected with the state/control boxes, and the mirror blocks
// linearised at the nominal.
void build_qp(const OrcProblem& P, int b, const double* xbar, const double* ubar,
              const double* A, const double* B, const double* d, double radius,
              double re, double rd, double rg, QP& qp) {
  const int N = P.N[b], nx = P.nx, nu = P.nu, n1 = nx + nu;
  qp.N = N; qp.nx = nx; qp.nu = nu; qp.maxblk = problem_maxblk(P);
  qp.rho_eq = re; qp.rho_dyn = rd; qp.rho_geo = rg;
  qp.xinit.assign(P.xinit + b * nx, P.xinit + (b + 1) * nx);
  qp.xtarget.assign(P.xtarget + b * nx, P.xtarget + (b + 1) * nx);
  qp.tmask.assign(P.tmask + b * nx, P.tmask + (b + 1) * nx);
  qp.node.assign(N + 1, QPNode());
  const double* Qd = P.Qd + b * nx; const double* xr = P.xref + b * nx;
  const double* Rd = P.Rd + b * nu; const double* ur = P.uref + b * nu;
  const double* QNd = P.QNd + b * nx; const double* qN = P.qN + b * nx;
  for (int i = 0; i <= N; ++i) {
    QPNode& nd = qp.node[i];
    const bool term = (i == N);
    nd.Q.assign(nx * nx, 0.0); nd.q.assign(nx, 0.0);
    for (int j = 0; j < nx; ++j) {
      const double w = term ? QNd[j] : Qd[j];
      nd.Q[j * nx + j] = w;
      nd.q[j] = -w * xr[j] + (term ? qN[j] : 0.0);
    }
    nd.xlo.resize(nx); nd.xhi.resize(nx);
    for (int j = 0; j < nx; ++j) {
      const double xb = xbar[i * nx + j];
      nd.xlo[j] = std::max(P.xlo[b * nx + j], xb - radius);
      nd.xhi[j] = std::min(P.xhi[b * nx + j], xb + radius);
    }
    if (!term) {
      nd.A.assign(A + (size_t)i * nx * nx, A + (size_t)(i + 1) * nx * nx);
      nd.B.assign(B + (size_t)i * nx * nu, B + (size_t)(i + 1) * nx * nu);
      nd.d.assign(d + (size_t)i * nx, d + (size_t)(i + 1) * nx);
      nd.R.assign(nu * nu, 0.0); nd.r.assign(nu, 0.0); nd.M.assign(nx * nu, 0.0);
      for (int j = 0; j < nu; ++j) { nd.R[j * nu + j] = Rd[j]; nd.r[j] = -Rd[j] * ur[j]; }
      nd.ulo.resize(nu); nd.uhi.resize(nu);
      for (int j = 0; j < nu; ++j) {
        const double ub = ubar[i * nu + j];
        nd.ulo[j] = std::max(P.ulo[b * nu + j], ub - radius);
        nd.uhi[j] = std::min(P.uhi[b * nu + j], ub + radius);
      }
    }
    const int n = term ? nx : n1;
    nd.blk.assign(qp.maxblk, Block());
    for (Block& bl : nd.blk) bl.G.assign(3 * n, 0.0);
    if (P.model == MODEL_MARS14) {
      const double* st = &P.sets[b * 8];
      // [0] |T| >= T_min (linearised), [1] |T| <= T_max, [2] tan of the glide-slope
      // half-angle from Up, [3] tan of the gimbal angle, [4] radius of (qy, qz)
      // (sin of half the largest tilt), [5] largest body rate
      if (st[2] > 0.0) {  // glide-slope cone on r (t = Up)
        Block& bl = nd.blk[0]; bl.kind = BLK_CONE; bl.p0 = st[2];
        for (int k = 0; k < 3; ++k) bl.G[k * n + 1 + k] = 1.0;
      }
      if (st[4] > 0.0) {  // tilt: |(qy, qz)| <= sin(theta_max / 2) (third row zero)
        Block& bl = nd.blk[1]; bl.kind = BLK_BALL; bl.p0 = st[4];
        bl.G[0 * n + 9] = 1.0; bl.G[1 * n + 10] = 1.0;
      }
      if (st[5] > 0.0) {  // |omega| <= omega_max
        Block& bl = nd.blk[2]; bl.kind = BLK_BALL; bl.p0 = st[5];
        for (int k = 0; k < 3; ++k) bl.G[k * n + 11 + k] = 1.0;
      }
      if (!term && st[1] > 0.0) {  // |T| <= T_max
        Block& bl = nd.blk[3]; bl.kind = BLK_BALL; bl.p0 = st[1];
        for (int k = 0; k < 3; ++k) bl.G[k * n + nx + k] = 1.0;
      }
      if (!term && st[0] > 0.0) {  // |T| >= T_min linearised at the nominal thrust
        const double* ub = &ubar[i * nu];
        double nv[3] = {ub[0], ub[1], ub[2]};
        double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        if (nn < 1e-12) { nv[0] = 1; nv[1] = 0; nv[2] = 0; nn = 1; }
        Block& bl = nd.blk[4]; bl.kind = BLK_HALF; bl.p0 = st[0];
        for (int k = 0; k < 3; ++k) bl.G[nx + k] = nv[k] / nn;
      }
      if (!term && st[3] > 0.0) {  // gimbal: |(T_y, T_z)| <= tan(delta_max) T_x
        Block& bl = nd.blk[5]; bl.kind = BLK_CONE; bl.p0 = st[3];
        for (int k = 0; k < 3; ++k) bl.G[k * n + nx + k] = 1.0;
      }
    } else if (P.model != MODEL_MARS7) {
      // Obstacle j, linearised about the nominal position:
      // n = (p - c)/|p - c|, keep n^T p >= n^T c + r (tie-break n = e_z).
      const double* p = &xbar[i * nx];
      for (int j = 0; j < P.nobs[b]; ++j) {
        const double* c = &P.obs_c[((size_t)b * P.max_obs + j) * 3];
        const double r = P.obs_r[(size_t)b * P.max_obs + j];
        double nv[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
        double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        if (nn < 1e-12) { nv[0] = 0; nv[1] = 0; nv[2] = 1; nn = 1; }
        Block& bl = nd.blk[j];
        bl.kind = BLK_HALF;
        for (int k = 0; k < 3; ++k) bl.G[k] = nv[k] / nn;
        bl.p0 = bl.G[0] * c[0] + bl.G[1] * c[1] + bl.G[2] * c[2] + r;
      }
    } else {
      const double* st = &P.sets[b * 8];
      if (st[2] > 0.0) {  // glide-slope cone on the position (t = Up)
        Block& bl = nd.blk[0]; bl.kind = BLK_CONE; bl.p0 = st[2];
        for (int k = 0; k < 3; ++k) bl.G[k * n + k] = 1.0;
      }
      if (!term && st[1] > 0.0) {  // |T| <= T_max
        Block& bl = nd.blk[1]; bl.kind = BLK_BALL; bl.p0 = st[1];
        for (int k = 0; k < 3; ++k) bl.G[k * n + nx + k] = 1.0;
      }
      if (!term && st[0] > 0.0) {  // |T| >= T_min linearised: (T_bar/|T_bar|)^T T >= T_min
        const double* ub = &ubar[i * nu];
        double nv[3] = {ub[0], ub[1], ub[2]};
        double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        if (nn < 1e-12) { nv[0] = 1; nv[1] = 0; nv[2] = 0; nn = 1; }
        Block& bl = nd.blk[2]; bl.kind = BLK_HALF; bl.p0 = st[0];
        for (int k = 0; k < 3; ++k) bl.G[nx + k] = nv[k] / nn;
      }
    }
  }
}

// Nonlinear cost phi(x_N) + sum l(x_i, u_i) of Eq. (1a) with the quadratic
// running/terminal costs of the workloads.
double traj_cost(const OrcProblem& P, int b, const double* x, const double* u) {
  const int N = P.N[b], nx = P.nx, nu = P.nu;
  const double* Qd = P.Qd + b * nx; const double* xr = P.xref + b * nx;
  const double* Rd = P.Rd + b * nu; const double* ur = P.uref + b * nu;
  double c = 0.0;
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < nx; ++j) { const double e = x[i * nx + j] - xr[j]; c += 0.5 * Qd[j] * e * e; }
    for (int j = 0; j < nu; ++j) { const double e = u[i * nu + j] - ur[j]; c += 0.5 * Rd[j] * e * e; }
  }
  for (int j = 0; j < nx; ++j) {
    const double e = x[N * nx + j] - xr[j];
    c += 0.5 * P.QNd[b * nx + j] * e * e + P.qN[b * nx + j] * x[N * nx + j];
  }
  return c;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- pins API
int orc_state_size(int N, int nx, int nu, int maxblk) { return (int)state_size(N, nx, nu, maxblk); }

void orc_f(int model, const double* prm, const double* x, const double* u, double* xd) {
  f_eval<double>(model, prm, x, u, xd);
}

void orc_rk4(int model, const double* prm, double h, const double* x, const double* u, double* xn) {
  rk4<double>(model, prm, h, x, u, xn);
}

// A, B, d about (x, u): A = dRK4/dx, B = dRK4/du, d = RK4(x,u) - A x - B u (Eq. (2b)).
void orc_linearize(int model, const double* prm, double h, const double* x, const double* u,
                   double* A, double* B, double* d, double* xn) {
  const int nx = model_nx(model), nu = model_nu(model);
  rk4_variational(model, prm, h, x, u, xn, A, B);
  for (int r = 0; r < nx; ++r) {
    double acc = xn[r];
    for (int c = 0; c < nx; ++c) acc -= A[r * nx + c] * x[c];
    for (int c = 0; c < nu; ++c) acc -= B[r * nu + c] * u[c];
    d[r] = acc;
  }
}

// Complex-step derivative of the RK4 map (Squire & Trapp 1998): Im(F(z + i h e_j))/h.
void orc_jac_complex_step(int model, const double* prm, double h, const double* x, const double* u,
                          double* A, double* B) {
  typedef std::complex<double> C;
  const int nx = model_nx(model), nu = model_nu(model);
  const double eps = 1e-30;
  C xc[16], uc[16], out[16];
  for (int c = 0; c < nx + nu; ++c) {
    for (int j = 0; j < nx; ++j) xc[j] = C(x[j], (c == j) ? eps : 0.0);
    for (int j = 0; j < nu; ++j) uc[j] = C(u[j], (c == nx + j) ? eps : 0.0);
    rk4<C>(model, prm, h, xc, uc, out);
    for (int r = 0; r < nx; ++r) {
      if (c < nx) A[r * nx + c] = out[r].imag() / eps;
      else B[r * nu + (c - nx)] = out[r].imag() / eps;
    }
  }
}

void orc_project(int kind, int dim, double p0, const double* y, double* out) {
  proj_block(kind, dim, p0, y, out);
}

// Generic QP ADMM (used by the pins): explicit per-node data.
//   Q[N+1][nx][nx], R[N][nu][nu], M[N][nx][nu], q[N+1][nx], r[N][nu],
//   A[N][nx][nx], B[N][nx][nu], d[N][nx], boxes, boundary data,
//   blocks: kind[(N+1)*mb], G[(N+1)*mb][3][n_i] (n_i = nx+nu, or nx at N, padded to nx+nu), p0[(N+1)*mb].
// If warm == 0 the state is initialised from (xbar, ubar); else read from state_io.
// Returns 0 on success, 4 on a failed factorisation.
int orc_admm_qp(int N, int nx, int nu,
                const double* A, const double* B, const double* d,
                const double* Q, const double* R, const double* M, const double* q, const double* r,
                const double* xlo, const double* xhi, const double* ulo, const double* uhi,
                const double* xinit, const unsigned char* tmask, const double* xtarget,
                int mb, const int* kind, const double* G, const double* p0,
                double rho_eq, double rho_dyn, double rho_geo,
                int iters, int warm, const double* xbar, const double* ubar,
                double* state_io, double* stats2) {
  QP qp;
  qp.N = N; qp.nx = nx; qp.nu = nu; qp.maxblk = mb;
  qp.rho_eq = rho_eq; qp.rho_dyn = rho_dyn; qp.rho_geo = rho_geo;
  qp.xinit.assign(xinit, xinit + nx);
  qp.xtarget.assign(xtarget, xtarget + nx);
  qp.tmask.assign(tmask, tmask + nx);
  qp.node.assign(N + 1, QPNode());
  const int n1 = nx + nu;
  for (int i = 0; i <= N; ++i) {
    QPNode& nd = qp.node[i];
    nd.Q.assign(Q + (size_t)i * nx * nx, Q + (size_t)(i + 1) * nx * nx);
    nd.q.assign(q + (size_t)i * nx, q + (size_t)(i + 1) * nx);
    nd.xlo.assign(xlo + (size_t)i * nx, xlo + (size_t)(i + 1) * nx);
    nd.xhi.assign(xhi + (size_t)i * nx, xhi + (size_t)(i + 1) * nx);
    if (i < N) {
      nd.A.assign(A + (size_t)i * nx * nx, A + (size_t)(i + 1) * nx * nx);
      nd.B.assign(B + (size_t)i * nx * nu, B + (size_t)(i + 1) * nx * nu);
      nd.d.assign(d + (size_t)i * nx, d + (size_t)(i + 1) * nx);
      nd.R.assign(R + (size_t)i * nu * nu, R + (size_t)(i + 1) * nu * nu);
      nd.M.assign(M + (size_t)i * nx * nu, M + (size_t)(i + 1) * nx * nu);
      nd.r.assign(r + (size_t)i * nu, r + (size_t)(i + 1) * nu);
      nd.ulo.assign(ulo + (size_t)i * nu, ulo + (size_t)(i + 1) * nu);
      nd.uhi.assign(uhi + (size_t)i * nu, uhi + (size_t)(i + 1) * nu);
    }
    const int n = (i < N) ? n1 : nx;
    nd.blk.assign(mb, Block());
    for (int b = 0; b < mb; ++b) {
      Block& bl = nd.blk[b];
      bl.kind = kind[i * mb + b];
      bl.p0 = p0[i * mb + b];
      bl.G.assign(3 * n, 0.0);
      for (int k = 0; k < 3; ++k)
        for (int c = 0; c < n; ++c) bl.G[k * n + c] = G[(((size_t)i * mb + b) * 3 + k) * n1 + c];
    }
  }
  State st;
  if (warm) { st.alloc(N, nx, nu, mb); st.from_flat(state_io); }
  else init_state(qp, xbar, ubar, st);
  AdmmStats s = admm_run(qp, st, iters);
  st.to_flat(state_io);
  if (stats2) { stats2[0] = s.primal; stats2[1] = s.dual; }
  return s.ok ? 0 : ST_NUMERIC;
}

// One ADMM call on the SCP's own QP for instance b (the unit the CUDA
// path's standalone ADMM entry point is checked against).  A, B, d are the
// instance's linearisation (A[N][nx][nx], ...), radius the trust region.
int orc_problem_admm(const OrcProblem* P, int b, const double* xbar, const double* ubar,
                     const double* A, const double* B, const double* d, double radius,
                     int iters, int warm, double* state_io, double* stats2) {
  QP qp;
  build_qp(*P, b, xbar, ubar, A, B, d, radius, P->rho_eq, P->rho_dyn, P->rho_geo, qp);
  State st;
  if (warm) { st.alloc(qp.N, qp.nx, qp.nu, qp.maxblk); st.from_flat(state_io); }
  else init_state(qp, xbar, ubar, st);
  AdmmStats s = admm_run(qp, st, iters);
  st.to_flat(state_io);
  if (stats2) { stats2[0] = s.primal; stats2[1] = s.dual; }
  return s.ok ? 0 : ST_NUMERIC;
}

// Per-instance result record (doubles):
//  0 defect_max of the returned trajectory   1 cost   2 merit J
//  3 primal residual   4 dual residual (last ADMM call)   5 trust radius
//  6 last step |cand - nominal|_inf   7 SCP iterations run   8 accepted count
//  9 accept bitmask (bit k = iteration k accepted)   10 status
enum { NSTAT = 16 };
// Per-iteration log (doubles, 8 per iteration):
//  0 accept  1 ratio (NaN if the model decrease is <= 1e-12)  2 J(nominal)
//  3 J(candidate)  4 L(candidate)  5 candidate max defect  6 radius after  7 step
enum { NLOG = 8 };

// SCP with fixed iteration counts or the stop test (Sec. III-A), one
// instance.  Acceptance (omitted by the paper): l1 merit
// J = cost + w_d sum |f(x_i,u_i) - x_{i+1}|_1, its linear model L with
// A x + B u + d in place of f; ratio = (J(x_bar) - J(cand)) / (J(x_bar) - L(cand));
// accept if ratio > 0 or the model decrease is <= 1e-12; radius halves below
// 0.25, doubles (capped) above 0.75, floored at tr_min.
//
// run_iters > 0: run exactly that many iterations (at most scp_iters) without
// the stop test -- the trajectory after a given iteration count, for comparing
// solves whose stop tests landed on opposite sides of defect_tol.  The penalty
// schedule stays that of the scp_iters cap.
//
// state0 (not NULL): the solve starts from that ADMM state (the flat absolute
// layout of orc_state_size) instead of the cold start -- a warm start from kept
// ADMM state (Sec. III-B warm-starts the inner solves); its mirrors are
// re-projected with the first QP's sets, as every later iteration does, and
// the penalties stay at the schedule's final value, at which a kept state was
// computed (the schedule of Sec. IV-A rises over a solve from a cold start).
void scp_instance(const OrcProblem& P, int b, const double* xg, const double* ug,
                  double* xout, double* uout, double* stat, double* log, int run_iters = 0,
                  const double* state0 = nullptr) {
  const int N = P.N[b], nx = P.nx, nu = P.nu;
  const double* prm = P.params + b * 8;
  const double h = P.dt[b];
  std::vector<double> xbar(xg, xg + (N + 1) * nx), ubar(ug, ug + N * nu);
  std::vector<double> A(N * nx * nx), B(N * nx * nu), d(N * nx), fnom(N * nx), fc(nx);
  double radius = P.tr_init;
  State st;
  int status = ST_OK, accepted = 0, iters_run = 0;
  double mask = 0.0, last_step = 0.0;
  AdmmStats as;
  const int K = P.scp_iters;
  for (int k = 0; k < K; ++k) {
    if (run_iters > 0 && k >= run_iters) break;
    // a warm start continues at the schedule's final penalty (its state was computed there)
    const int ks = state0 ? K - 1 : k;
    double fac = 1.0;
    if (P.rho_final > 0.0 && K > 1) fac = std::pow(P.rho_final / P.rho_geo, (double)ks / (K - 1));
    const double re = P.rho_eq * fac, rd = P.rho_dyn * fac, rg = P.rho_geo * fac;
    for (int i = 0; i < N; ++i)
      orc_linearize(P.model, prm, h, &xbar[i * nx], &ubar[i * nu], &A[i * nx * nx], &B[i * nx * nu],
                    &d[i * nx], &fnom[i * nx]);
    QP qp;
    build_qp(P, b, xbar.data(), ubar.data(), A.data(), B.data(), d.data(), radius, re, rd, rg, qp);
    if (k == 0 && !state0) {
      init_state(qp, xbar.data(), ubar.data(), st);
    } else {
      if (k == 0) { st.alloc(qp.N, qp.nx, qp.nu, qp.maxblk); st.from_flat(state0); }
      reseed_mirrors(qp, st);
    }
    as = admm_run(qp, st, P.admm_iters);
    ++iters_run;
    if (!as.ok) { status = ST_NUMERIC; break; }
    // candidate = the mirror pair (x-hat, u-hat)
    const std::vector<double>& xc = st.xh;
    const std::vector<double>& uc = st.uh;
    double nl_nom = 0.0, nl_c = 0.0, lin_c = 0.0, dmax_c = 0.0, step = 0.0;
    for (int i = 0; i < N; ++i) {
      rk4<double>(P.model, prm, h, &xc[i * nx], &uc[i * nu], fc.data());
      double dinf = 0.0;
      for (int j = 0; j < nx; ++j) {
        nl_nom += std::fabs(fnom[i * nx + j] - xbar[(i + 1) * nx + j]);
        const double e = fc[j] - xc[(i + 1) * nx + j];
        nl_c += std::fabs(e);
        dinf = std::max(dinf, std::fabs(e));
        double lin = d[i * nx + j];
        for (int c = 0; c < nx; ++c) lin += A[(i * nx + j) * nx + c] * xc[i * nx + c];
        for (int c = 0; c < nu; ++c) lin += B[(i * nx + j) * nu + c] * uc[i * nu + c];
        lin_c += std::fabs(lin - xc[(i + 1) * nx + j]);
      }
      dmax_c = std::max(dmax_c, dinf);
    }
    for (int e = 0; e < (N + 1) * nx; ++e) step = std::max(step, std::fabs(xc[e] - xbar[e]));
    for (int e = 0; e < N * nu; ++e) step = std::max(step, std::fabs(uc[e] - ubar[e]));
    const double cn = traj_cost(P, b, xbar.data(), ubar.data());
    const double cc = traj_cost(P, b, xc.data(), uc.data());
    const double Jn = cn + P.w_d * nl_nom, Jc = cc + P.w_d * nl_c, Lc = cc + P.w_d * lin_c;
    const double den = Jn - Lc, num = Jn - Jc;
    bool accept;
    double ratio = NAN;
    if (den <= 1e-12) {
      accept = true;
    } else {
      ratio = num / den;
      accept = ratio > 0.0;
      if (ratio < 0.25) radius *= 0.5;
      else if (ratio > 0.75) radius = std::min(2.0 * radius, P.tr_max);
    }
    radius = std::max(radius, P.tr_min);
    if (!std::isfinite(Jc)) { accept = false; status = ST_NUMERIC; }
    if (accept) {
      xbar = xc; ubar = uc;
      ++accepted;
      mask += std::ldexp(1.0, k);
    }
    last_step = step;
    if (log) {
      double* L = &log[((size_t)b * K + k) * NLOG];
      L[0] = accept; L[1] = ratio; L[2] = Jn; L[3] = Jc; L[4] = Lc; L[5] = dmax_c; L[6] = radius; L[7] = step;
    }
    if (status == ST_NUMERIC) break;
    if (run_iters <= 0 && P.stop && accept && dmax_c <= P.defect_tol && step <= P.step_tol) break;
  }
  // defect of the returned (last accepted) trajectory
  double dmax = 0.0, nl = 0.0;
  for (int i = 0; i < N; ++i) {
    rk4<double>(P.model, prm, h, &xbar[i * nx], &ubar[i * nu], fc.data());
    for (int j = 0; j < nx; ++j) {
      const double e = std::fabs(fc[j] - xbar[(i + 1) * nx + j]);
      dmax = std::max(dmax, e);
      nl += e;
    }
  }
  if (!std::isfinite(dmax)) status = ST_NUMERIC;
  if (status == ST_OK && !(dmax <= P.defect_tol)) status = ST_NOTCONV;
  std::copy(xbar.begin(), xbar.end(), xout);
  std::copy(ubar.begin(), ubar.end(), uout);
  const double c = traj_cost(P, b, xbar.data(), ubar.data());
  double* S = &stat[(size_t)b * NSTAT];
  for (int j = 0; j < NSTAT; ++j) S[j] = 0.0;
  S[0] = dmax; S[1] = c; S[2] = c + P.w_d * nl; S[3] = as.primal; S[4] = as.dual;
  S[5] = radius; S[6] = last_step; S[7] = iters_run; S[8] = accepted; S[9] = mask; S[10] = status;
}

// Non-anticipativity of the robust MPC (Sec. IV-A): after Step 3 the first
// control mirror of every scenario becomes the projection of the scenarios'
// Step-3 arguments u_0 + nu_u,0 / rho_geo onto {u_0^(1) = ... = u_0^(K)}
// intersected with every scenario's box -- the clamped average.
void consensus_u0(const std::vector<QP>& qps, std::vector<State>& sts) {
  const int K = (int)qps.size(), nu = qps[0].nu;
  const double rg = qps[0].rho_geo;
  for (int j = 0; j < nu; ++j) {
    double sum = 0.0, lo = -INFINITY, hi = INFINITY;
    for (int k = 0; k < K; ++k) {
      sum += sts[k].u[j] + sts[k].nuu[j] / rg;
      lo = std::max(lo, qps[k].node[0].ulo[j]);
      hi = std::min(hi, qps[k].node[0].uhi[j]);
    }
    const double v = std::min(std::max(sum / K, lo), hi);
    for (int k = 0; k < K; ++k) sts[k].uh[j] = v;
  }
}

// SCP of one group of K scenarios (instances b0 .. b0+K-1) sharing the first
// control.  The scenarios' ADMM iterations run in lockstep with the consensus
// step between Step 3 and Step 4; the acceptance test is taken on the group
// (sums of merit and model over the scenarios, one trust radius, one
// decision), so accepted nominals keep a common first control.
// run_iters > 0: exactly that many iterations without the stop test (as scp_instance).
void scp_group(const OrcProblem& P, int b0, int K, const double* xg_all, const double* ug_all,
               double* xout_all, double* uout_all, double* stat, double* log, int run_iters = 0) {
  const int nx = P.nx, nu = P.nu;
  std::vector<std::vector<double>> xbar(K), ubar(K), A(K), B(K), d(K), fnom(K);
  std::vector<QP> qps(K);
  std::vector<State> sts(K);
  std::vector<AdmmWork> wks(K);
  std::vector<AdmmStats> ass(K);
  for (int k = 0; k < K; ++k) {
    const int b = b0 + k, N = P.N[b];
    xbar[k].assign(xg_all + P.xoff[b] * nx, xg_all + (P.xoff[b] + N + 1) * nx);
    ubar[k].assign(ug_all + P.uoff[b] * nu, ug_all + (P.uoff[b] + N) * nu);
    A[k].resize(N * nx * nx); B[k].resize(N * nx * nu); d[k].resize(N * nx); fnom[k].resize(N * nx);
  }
  double radius = P.tr_init, mask = 0.0, last_step = 0.0;
  int status = ST_OK, accepted = 0, iters_run = 0;
  const int Kscp = P.scp_iters;
  std::vector<double> fc(nx);
  for (int it_scp = 0; it_scp < Kscp; ++it_scp) {
    if (run_iters > 0 && it_scp >= run_iters) break;
    double fac = 1.0;
    if (P.rho_final > 0.0 && Kscp > 1) fac = std::pow(P.rho_final / P.rho_geo, (double)it_scp / (Kscp - 1));
    const double re = P.rho_eq * fac, rd = P.rho_dyn * fac, rg = P.rho_geo * fac;
    bool ok = true;
    for (int k = 0; k < K; ++k) {
      const int b = b0 + k, N = P.N[b];
      const double* prm = P.params + b * 8;
      for (int i = 0; i < N; ++i)
        orc_linearize(P.model, prm, P.dt[b], &xbar[k][i * nx], &ubar[k][i * nu], &A[k][i * nx * nx],
                      &B[k][i * nx * nu], &d[k][i * nx], &fnom[k][i * nx]);
      build_qp(P, b, xbar[k].data(), ubar[k].data(), A[k].data(), B[k].data(), d[k].data(), radius, re, rd, rg, qps[k]);
      if (it_scp == 0) init_state(qps[k], xbar[k].data(), ubar[k].data(), sts[k]);
      else reseed_mirrors(qps[k], sts[k]);
      ok = admm_prepare(qps[k], wks[k]) && ok;
    }
    ++iters_run;
    if (!ok) { status = ST_NUMERIC; break; }
    for (int it = 0; it < P.admm_iters; ++it) {
      const bool last = (it == P.admm_iters - 1);
      for (int k = 0; k < K; ++k) admm_first_part(qps[k], sts[k], wks[k], last);
      consensus_u0(qps, sts);
      for (int k = 0; k < K; ++k) admm_second_part(qps[k], sts[k], wks[k], last, ass[k]);
    }
    double Jn = 0.0, Jc = 0.0, Lc = 0.0, dmax = 0.0, step = 0.0;
    std::vector<double> dmax_k(K, 0.0);
    for (int k = 0; k < K; ++k) {
      const int b = b0 + k, N = P.N[b];
      const double* prm = P.params + b * 8;
      const std::vector<double>& xc = sts[k].xh;
      const std::vector<double>& uc = sts[k].uh;
      double nl_nom = 0.0, nl_c = 0.0, lin_c = 0.0;
      for (int i = 0; i < N; ++i) {
        rk4<double>(P.model, prm, P.dt[b], &xc[i * nx], &uc[i * nu], fc.data());
        for (int j = 0; j < nx; ++j) {
          nl_nom += std::fabs(fnom[k][i * nx + j] - xbar[k][(i + 1) * nx + j]);
          const double e = fc[j] - xc[(i + 1) * nx + j];
          nl_c += std::fabs(e);
          dmax_k[k] = std::max(dmax_k[k], std::fabs(e));
          double lin = d[k][i * nx + j];
          for (int c = 0; c < nx; ++c) lin += A[k][(i * nx + j) * nx + c] * xc[i * nx + c];
          for (int c = 0; c < nu; ++c) lin += B[k][(i * nx + j) * nu + c] * uc[i * nu + c];
          lin_c += std::fabs(lin - xc[(i + 1) * nx + j]);
        }
      }
      for (size_t e = 0; e < xc.size(); ++e) step = std::max(step, std::fabs(xc[e] - xbar[k][e]));
      for (size_t e = 0; e < uc.size(); ++e) step = std::max(step, std::fabs(uc[e] - ubar[k][e]));
      const double cn = traj_cost(P, b, xbar[k].data(), ubar[k].data());
      const double cc = traj_cost(P, b, xc.data(), uc.data());
      Jn += cn + P.w_d * nl_nom; Jc += cc + P.w_d * nl_c; Lc += cc + P.w_d * lin_c;
      dmax = std::max(dmax, dmax_k[k]);
    }
    const double den = Jn - Lc, num = Jn - Jc;
    bool accept;
    double ratio = NAN;
    if (den <= 1e-12) {
      accept = true;
    } else {
      ratio = num / den;
      accept = ratio > 0.0;
      if (ratio < 0.25) radius *= 0.5;
      else if (ratio > 0.75) radius = std::min(2.0 * radius, P.tr_max);
    }
    radius = std::max(radius, P.tr_min);
    if (!std::isfinite(Jc)) { accept = false; status = ST_NUMERIC; }
    if (accept) {
      for (int k = 0; k < K; ++k) { xbar[k] = sts[k].xh; ubar[k] = sts[k].uh; }
      ++accepted;
      mask += std::ldexp(1.0, it_scp);
    }
    last_step = step;
    if (log)
      for (int k = 0; k < K; ++k) {
        double* L = &log[((size_t)(b0 + k) * Kscp + it_scp) * NLOG];
        L[0] = accept; L[1] = ratio; L[2] = Jn; L[3] = Jc; L[4] = Lc; L[5] = dmax; L[6] = radius; L[7] = step;
      }
    if (status == ST_NUMERIC) break;
    if (run_iters <= 0 && P.stop && accept && dmax <= P.defect_tol && step <= P.step_tol) break;
  }
  for (int k = 0; k < K; ++k) {
    const int b = b0 + k, N = P.N[b];
    const double* prm = P.params + b * 8;
    double dm = 0.0, nl = 0.0;
    for (int i = 0; i < N; ++i) {
      rk4<double>(P.model, prm, P.dt[b], &xbar[k][i * nx], &ubar[k][i * nu], fc.data());
      for (int j = 0; j < nx; ++j) {
        const double e = std::fabs(fc[j] - xbar[k][(i + 1) * nx + j]);
        dm = std::max(dm, e);
        nl += e;
      }
    }
    int st = status;
    if (!std::isfinite(dm)) st = ST_NUMERIC;
    if (st == ST_OK && !(dm <= P.defect_tol)) st = ST_NOTCONV;
    std::copy(xbar[k].begin(), xbar[k].end(), xout_all + P.xoff[b] * nx);
    std::copy(ubar[k].begin(), ubar[k].end(), uout_all + P.uoff[b] * nu);
    const double c = traj_cost(P, b, xbar[k].data(), ubar[k].data());
    double* S = &stat[(size_t)b * NSTAT];
    for (int j = 0; j < NSTAT; ++j) S[j] = 0.0;
    S[0] = dm; S[1] = c; S[2] = c + P.w_d * nl; S[3] = ass[k].primal; S[4] = ass[k].dual;
    S[5] = radius; S[6] = last_step; S[7] = iters_run; S[8] = accepted; S[9] = mask; S[10] = st;
  }
}

// Solve every instance; xout/uout packed like the guesses.  nthreads <= 0: OpenMP default.
int orc_scp_solve(const OrcProblem* P, const double* xg, const double* ug, double* xout, double* uout,
                  double* stat, double* log, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < P->batch; ++b) {
    if (P->group > 1) {
      if (b % P->group == 0) scp_group(*P, b, P->group, xg, ug, xout, uout, stat, log);
      continue;
    }
    const long long xo = P->xoff[b], uo = P->uoff[b];
    scp_instance(*P, b, xg + xo * P->nx, ug + uo * P->nu, xout + xo * P->nx, uout + uo * P->nu, stat, log);
  }
  return 0;
}

// Every instance (or scenario group, by its first instance's entry) solved
// with exactly run_iters[b] SCP iterations (no stop test; see scp_instance);
// run_iters[b] <= 0 keeps the stop test.
int orc_scp_solve_iters(const OrcProblem* P, const double* xg, const double* ug, double* xout, double* uout,
                        double* stat, const int* run_iters, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < P->batch; ++b) {
    if (P->group > 1) {
      if (b % P->group == 0) scp_group(*P, b, P->group, xg, ug, xout, uout, stat, nullptr, run_iters[b]);
      continue;
    }
    const long long xo = P->xoff[b], uo = P->uoff[b];
    scp_instance(*P, b, xg + xo * P->nx, ug + uo * P->nu, xout + xo * P->nx, uout + uo * P->nu, stat, nullptr,
                 run_iters[b]);
  }
  return 0;
}

// Independent instances solved from given ADMM states (state_all: each
// instance's flat state, instances one after the other in batch order).
int orc_scp_solve_warm(const OrcProblem* P, const double* xg, const double* ug, const double* state_all,
                       double* xout, double* uout, double* stat, int nthreads) {
  if (P->group > 1) return 1;
  std::vector<long long> so(P->batch + 1, 0);
  const int mb = P->model == 1 || P->model == 3 ? P->max_obs : (P->model == 4 ? 6 : 3);
  for (int b = 0; b < P->batch; ++b) so[b + 1] = so[b] + orc_state_size(P->N[b], P->nx, P->nu, mb);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int b = 0; b < P->batch; ++b) {
    const long long xo = P->xoff[b], uo = P->uoff[b];
    scp_instance(*P, b, xg + xo * P->nx, ug + uo * P->nu, xout + xo * P->nx, uout + uo * P->nu, stat, nullptr, 0,
                 state_all + so[b]);
  }
  return 0;
}

// Max defect max_i |RK4(x_i, u_i) - x_{i+1}|_inf (Eq. (1b)) of every instance
// of packed trajectories x, u (laid out like the guesses), in FP64.
int orc_traj_defects(const OrcProblem* P, const double* x, const double* u, double* out) {
  const int nx = P->nx, nu = P->nu;
  for (int b = 0; b < P->batch; ++b) {
    const long long xo = P->xoff[b], uo = P->uoff[b];
    std::vector<double> f(nx);
    double m = 0.0;
    for (int i = 0; i < P->N[b]; ++i) {
      rk4<double>(P->model, P->params + b * 8, P->dt[b], x + (xo + i) * nx, u + (uo + i) * nu, f.data());
      for (int j = 0; j < nx; ++j) m = std::max(m, std::fabs(f[j] - x[(xo + i + 1) * nx + j]));
    }
    out[b] = m;
  }
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
