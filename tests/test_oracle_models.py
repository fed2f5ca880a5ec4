"""Pins of the oracle's dynamics, RK4 step and linearisation (Eq. (1b), (2b)).

Each test ties the oracle to something other than itself: closed-form
motions, conservation laws, the matrix exponential of a constant body rate,
RK4's order, and complex-step / finite-difference derivatives.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
import workloads as W

QUAD = W.MODEL_QUAD12
MARS = W.MODEL_MARS7
QUAT = W.MODEL_QUAT13
MARS6 = W.MODEL_MARS14


def quad_params(m=1.0, J=(0.01, 0.01, 0.02), l=0.2, km=0.01, cd=0.0, g=9.81):
    return np.array([m, *J, l, km, cd, g, ])


def mars_params():
    p = W.mars_batch(1)
    return p.params[0]


def mars6_params():
    return W.mars6_batch(1).params[0]


def rollout(model, prm, h, x, u, steps):
    for _ in range(steps):
        x = oracle.rk4(model, prm, h, x, u)
    return x


def R_zyx(phi, th, psi):
    cx, sx, cy, sy, cz, sz = math.cos(phi), math.sin(phi), math.cos(th), math.sin(th), math.cos(psi), math.sin(psi)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def quat_mul(a, b):
    """Hamilton product, scalar first."""
    return np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                     a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                     a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                     a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])


def quat_from_euler(phi, th, psi):
    """q of R = Rz(psi) Ry(theta) Rx(phi): q = qz (x) qy (x) qx."""
    qx = np.array([math.cos(phi / 2), math.sin(phi / 2), 0, 0])
    qy = np.array([math.cos(th / 2), 0, math.sin(th / 2), 0])
    qz = np.array([math.cos(psi / 2), 0, 0, math.sin(psi / 2)])
    return quat_mul(qz, quat_mul(qy, qx))


# ------------------------------------------------------------------ quadrotor
def test_quad_hover_is_equilibrium():
    prm = quad_params()
    x = np.zeros(12); x[0:3] = [1.0, -2.0, 3.0]; x[8] = 0.7   # any position and yaw
    u = np.full(4, 9.81 / 4)
    np.testing.assert_allclose(oracle.f(QUAD, prm, x, u), 0.0, atol=1e-15)
    np.testing.assert_allclose(oracle.rk4(QUAD, prm, 0.05, x, u), x, atol=1e-15)


def test_quad_vertical_climb_closed_form():
    # level attitude, thrust 2mg: constant upward acceleration g; RK4 is exact on quadratics
    prm = quad_params(m=1.3)
    u = np.full(4, 2 * 1.3 * 9.81 / 4)
    x = rollout(QUAD, prm, 0.05, np.zeros(12), u, 40)
    t = 2.0
    assert abs(x[2] - 0.5 * 9.81 * t * t) < 1e-10
    assert abs(x[5] - 9.81 * t) < 1e-11
    np.testing.assert_allclose(x[[0, 1, 3, 4, 6, 7, 8, 9, 10, 11]], 0.0, atol=1e-12)


def test_quad_drag_is_exponential_decay():
    # hover thrust, level, drag cd: v' = -(cd/m) v (horizontal), so v(t) = v0 exp(-cd t/m)
    cd, m = 0.2, 0.9
    prm = quad_params(m=m, cd=cd)
    x = np.zeros(12); x[3] = 1.5
    xt = rollout(QUAD, prm, 0.01, x, np.full(4, m * 9.81 / 4), 200)
    assert abs(xt[3] - 1.5 * math.exp(-cd * 2.0 / m)) < 1e-10
    assert abs(xt[0] - 1.5 * m / cd * (1 - math.exp(-cd * 2.0 / m))) < 1e-10


def test_quad_roll_tilts_thrust_toward_minus_y():
    # positive roll phi rotates the body z-axis to (0, -sin phi, cos phi) (R = Rz Ry Rx)
    prm = quad_params()
    x = np.zeros(12); x[6] = 0.3
    xd = oracle.f(QUAD, prm, x, np.full(4, 1.0))
    F = 4.0
    np.testing.assert_allclose(xd[3:6], [0.0, -math.sin(0.3) * F, math.cos(0.3) * F - 9.81], atol=1e-14)


def test_quad_attitude_kinematics_match_matrix_exponential():
    # isotropic inertia: a constant body rate stays constant, and R(t) = R(0) expm(t [w]x)
    prm = quad_params(J=(0.02, 0.02, 0.02))
    w = np.array([0.7, -0.4, 0.9])
    x = np.zeros(12); x[6:9] = [0.2, -0.3, 0.5]; x[9:12] = w
    u = np.full(4, 0.3)           # equal rotor thrusts: zero torque
    T, steps = 0.8, 800
    xt = rollout(QUAD, prm, T / steps, x, u, steps)
    R0 = R_zyx(*x[6:9])
    np.testing.assert_allclose(R_zyx(*xt[6:9]), R0 @ expm(T * hat(w)), atol=1e-10)
    np.testing.assert_allclose(xt[9:12], w, atol=1e-13)


def test_quad_torque_free_rotation_conserves_energy_and_momentum():
    # Euler's equations: 1/2 w^T J w and |J w| are invariants of torque-free motion
    J = np.array([0.01, 0.015, 0.02])
    prm = quad_params(J=tuple(J))
    x = np.zeros(12); x[9:12] = [1.0, 2.0, -1.5]
    xt = rollout(QUAD, prm, 1e-3, x, np.full(4, 0.2), 2000)
    w0, w1 = x[9:12], xt[9:12]
    assert abs(0.5 * w1 @ (J * w1) - 0.5 * w0 @ (J * w0)) < 1e-11
    assert abs(np.linalg.norm(J * w1) - np.linalg.norm(J * w0)) < 1e-11
    assert np.abs(w1 - w0).max() > 1e-2      # the motion is not trivial


def test_quad_rotor_torque_map():
    # "+" layout: rotor 2 vs 4 rolls, rotor 3 vs 1 pitches, (1,3) vs (2,4) yaws
    prm = quad_params()
    l, km, J = 0.2, 0.01, (0.01, 0.01, 0.02)
    for k, expect in enumerate([(0, -l, km), (l, 0, -km), (0, l, km), (-l, 0, -km)]):
        u = np.zeros(4); u[k] = 1.0
        wd = oracle.f(QUAD, prm, np.zeros(12), u)[9:12]
        np.testing.assert_allclose(wd, np.array(expect) / np.array(J), atol=1e-13)


# ------------------------------------------------------------------ Mars
def rocket_closed_form(prm, x0, T, t):
    """Constant thrust vector: Tsiolkovsky velocity and its integral."""
    g, alpha = prm[0], prm[1]
    Tn = np.linalg.norm(T); k = alpha * Tn; m0 = x0[6]
    m = m0 - k * t
    gv = np.array([-g, 0, 0]); e = T / Tn
    v = x0[3:6] + gv * t + e * (Tn / k) * math.log(m0 / m)
    I = t * math.log(m0) + ((m * math.log(m) - m) - (m0 * math.log(m0) - m0)) / k
    r = x0[0:3] + x0[3:6] * t + 0.5 * gv * t * t + e * (Tn / k) * I
    return np.concatenate([r, v, [m]])


def test_mars_constant_thrust_matches_rocket_equation():
    prm = mars_params()
    x0 = np.array([2.0, 0.3, -0.1, -0.6, 0.1, 0.05, 1.0])
    T = np.array([0.8, 0.2, -0.1])
    xt = rollout(MARS, prm, 0.01, x0, T, 600)
    np.testing.assert_allclose(xt, rocket_closed_form(prm, x0, T, 6.0), atol=1e-10, rtol=0)


def test_mars_free_fall():
    prm = mars_params()
    x0 = np.array([2.0, 0.3, -0.1, -0.6, 0.1, 0.05, 1.0])
    xt = rollout(MARS, prm, 0.06, x0, np.zeros(3), 100)
    t = 6.0
    np.testing.assert_allclose(xt[0], 2.0 - 0.6 * t - 0.5 * prm[0] * t * t, atol=1e-12)
    np.testing.assert_allclose(xt[1:3], x0[1:3] + x0[4:6] * t, atol=1e-12)
    assert xt[6] == 1.0


@pytest.mark.parametrize("model", [QUAD, MARS, QUAT])
def test_rk4_is_fourth_order(model):
    # one-step error against a converged fine rollout shrinks ~32x when h halves
    if model == QUAD:
        prm = quad_params(cd=0.1)
        x = np.array([0.1, 0.2, 0.3, 0.5, -0.4, 0.2, 0.3, -0.2, 0.4, 1.0, -2.0, 0.5])
        u = np.array([2.0, 3.0, 2.5, 1.5])
    elif model == QUAT:
        prm = quad_params(cd=0.1)
        x = np.concatenate([[0.1, 0.2, 0.3, 0.5, -0.4, 0.2], quat_from_euler(0.3, -0.2, 0.4), [1.0, -2.0, 0.5]])
        u = np.array([9.0, 0.05, -0.08, 0.02])
    else:
        prm = mars_params()
        x = np.array([2.0, 0.3, -0.1, -0.6, 0.1, 0.05, 1.0]); u = np.array([0.8, 0.2, -0.1])
    h = 0.2
    truth = {hh: rollout(model, prm, hh / 256, x, u, 256) for hh in (h, h / 2)}
    e1 = np.abs(oracle.rk4(model, prm, h, x, u) - truth[h]).max()
    e2 = np.abs(oracle.rk4(model, prm, h / 2, x, u) - truth[h / 2]).max()
    assert 24 < e1 / e2 < 40, e1 / e2


# ------------------------------------------------------------------ linearisation
def random_point(model, seed):
    rng = np.random.default_rng(seed)
    if model == QUAD:
        x = rng.uniform(-1, 1, 12); x[6:9] *= 0.6
        u = rng.uniform(0.5, 4.0, 4)
        prm = quad_params(cd=0.15)
    elif model == QUAT:
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        x = np.concatenate([rng.uniform(-1, 1, 6), q, rng.uniform(-2, 2, 3)])
        u = np.concatenate([rng.uniform(3, 15, 1), rng.uniform(-0.5, 0.5, 3)])
        prm = quad_params(cd=0.15)
    elif model == MARS6:
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        x = np.concatenate([[rng.uniform(0.8, 2.0)], rng.uniform(-1, 2, 6), q, rng.uniform(-0.5, 0.5, 3)])
        u = np.concatenate([rng.uniform(0.5, 2.5, 1), rng.uniform(-0.4, 0.4, 2)])
        prm = mars6_params()
    else:
        x = np.concatenate([rng.uniform(0.5, 2, 3), rng.uniform(-0.5, 0.5, 3), [rng.uniform(0.8, 1.0)]])
        u = rng.uniform(-0.6, 0.9, 3)
        prm = mars_params()
    return prm, x, u


@pytest.mark.parametrize("model", [QUAD, MARS, QUAT, MARS6])
@pytest.mark.parametrize("seed", range(5))
def test_jacobians_match_complex_step(model, seed):
    prm, x, u = random_point(model, seed)
    h = 0.05 if model == QUAD else 0.06
    A, B, d, xn = oracle.linearize(model, prm, h, x, u)
    Acs, Bcs = oracle.jac_complex_step(model, prm, h, x, u)
    np.testing.assert_allclose(A, Acs, atol=1e-13, rtol=1e-12)
    np.testing.assert_allclose(B, Bcs, atol=1e-13, rtol=1e-12)
    # the residual closes the affine model at the nominal: A x + B u + d = RK4(x, u)
    np.testing.assert_allclose(A @ x + B @ u + d, oracle.rk4(model, prm, h, x, u), atol=1e-14)
    np.testing.assert_allclose(xn, oracle.rk4(model, prm, h, x, u), atol=0)


@pytest.mark.parametrize("model", [QUAD, MARS, QUAT, MARS6])
def test_jacobians_match_central_differences(model):
    prm, x, u = random_point(model, 11)
    h = 0.05
    A, B, _, _ = oracle.linearize(model, prm, h, x, u)
    eps = 1e-6
    nx = x.size
    for j in range(nx + u.size):
        dz = np.zeros(nx + u.size); dz[j] = eps
        fp = oracle.rk4(model, prm, h, x + dz[:nx], u + dz[nx:])
        fm = oracle.rk4(model, prm, h, x - dz[:nx], u - dz[nx:])
        col = (fp - fm) / (2 * eps)
        ref = A[:, j] if j < nx else B[:, j - nx]
        np.testing.assert_allclose(col, ref, atol=2e-8)


# ------------------------------------------------------------------ 13-state quaternion quadrotor
def test_quat_hover_is_equilibrium_at_any_yaw():
    prm = quad_params()
    for psi in (0.0, 0.7, -2.5):
        x = np.concatenate([[1.0, -2.0, 3.0, 0, 0, 0], quat_from_euler(0, 0, psi), [0, 0, 0]])
        u = np.array([9.81, 0.0, 0.0, 0.0])
        np.testing.assert_allclose(oracle.f(QUAT, prm, x, u), 0.0, atol=1e-14)


def test_quat_matches_the_euler_model_under_the_rotor_map():
    # the 12-state Euler-angle model and the 13-state quaternion model describe the
    # same rigid body: with q = q(eta), T = sum f_i and tau = the rotor torque map,
    # accelerations agree, and q' is the chain rule of q(eta) along eta' = W omega
    rng = np.random.default_rng(3)
    prm = quad_params(cd=0.12)
    l, km = prm[4], prm[5]
    for _ in range(5):
        eta = rng.uniform(-0.6, 0.6, 3)
        p, v, w = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3), rng.uniform(-2, 2, 3)
        fr = rng.uniform(0.5, 4.0, 4)
        x12 = np.concatenate([p, v, eta, w])
        q = quat_from_euler(*eta)
        x13 = np.concatenate([p, v, q, w])
        u13 = np.array([fr.sum(), l * (fr[1] - fr[3]), l * (fr[2] - fr[0]), km * (fr[0] - fr[1] + fr[2] - fr[3])])
        d12 = oracle.f(QUAD, prm, x12, fr)
        d13 = oracle.f(QUAT, prm, x13, u13)
        np.testing.assert_allclose(d13[0:6], d12[0:6], atol=1e-13)
        np.testing.assert_allclose(d13[10:13], d12[9:12], atol=1e-12)
        eps = 1e-6
        dq = np.zeros(4)
        for k in range(3):
            e = np.zeros(3); e[k] = eps
            dq += (quat_from_euler(*(eta + e)) - quat_from_euler(*(eta - e))) / (2 * eps) * d12[6 + k]
        np.testing.assert_allclose(d13[6:10], dq, atol=1e-8)


def test_quat_thrust_direction_is_the_body_z_axis():
    prm = quad_params()
    for eta in ((0.3, -0.2, 0.4), (-0.5, 0.1, 2.0)):
        q = quat_from_euler(*eta)
        x = np.concatenate([np.zeros(6), q, np.zeros(3)])
        d = oracle.f(QUAT, prm, x, np.array([2.0, 0, 0, 0]))
        np.testing.assert_allclose(d[3:6] + np.array([0, 0, 9.81]), 2.0 * R_zyx(*eta)[:, 2], atol=1e-14)


def test_quat_kinematics_keep_the_norm_rate_zero():
    rng = np.random.default_rng(5)
    prm = quad_params()
    for _ in range(10):
        q = rng.normal(size=4) * rng.uniform(0.5, 2.0)
        x = np.concatenate([np.zeros(6), q, rng.uniform(-3, 3, 3)])
        d = oracle.f(QUAT, prm, x, np.array([5.0, 0.1, -0.2, 0.3]))
        assert abs(q @ d[6:10]) < 1e-14 * max(1.0, q @ q)


def test_quat_spin_about_a_principal_axis_matches_closed_form():
    prm = quad_params()
    wz = 1.3
    x = np.concatenate([np.zeros(6), [1, 0, 0, 0], [0, 0, wz]])
    u = np.array([9.81, 0, 0, 0])
    t = 2.0
    xt = rollout(QUAT, prm, 0.01, x, u, 200)
    np.testing.assert_allclose(xt[6:10], [math.cos(wz * t / 2), 0, 0, math.sin(wz * t / 2)], atol=1e-9)
    np.testing.assert_allclose(xt[10:13], [0, 0, wz], atol=1e-15)
    # hover thrust holds the body still up to the RK4 drift of |q| (thrust scales with |q|^2)
    np.testing.assert_allclose(xt[0:6], 0.0, atol=1e-8)


# ------------------------------------------------------------------ 14-state 6-DOF Mars
def rot_from_quat(q):
    from scipy.spatial.transform import Rotation
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()     # scipy: scalar last


def test_mars6_translation_and_mass_match_the_3dof_model_under_the_attitude():
    # with the body thrust rotated to the world frame by an independent rotation
    # matrix, (m, r, v) evolve exactly as the 3-DOF model's (r, v, m)
    rng = np.random.default_rng(4)
    p6, p3 = mars6_params(), mars_params().copy()
    p3[0], p3[1] = p6[1], p6[0]                      # same g and alpha
    for _ in range(5):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        m = rng.uniform(0.8, 2.0)
        r, v, w = rng.uniform(-1, 2, 3), rng.uniform(-1, 1, 3), rng.uniform(-0.5, 0.5, 3)
        TB = np.array([rng.uniform(0.5, 2.5), rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4)])
        d6 = oracle.f(MARS6, p6, np.concatenate([[m], r, v, q, w]), TB)
        d3 = oracle.f(MARS, p3, np.concatenate([r, v, [m]]), rot_from_quat(q) @ TB)
        np.testing.assert_allclose(d6[1:7], d3[0:6], atol=1e-14)
        np.testing.assert_allclose(d6[0], d3[6], atol=1e-15)


def test_mars6_attitude_and_rate_dynamics():
    rng = np.random.default_rng(8)
    prm = mars6_params()
    J = np.diag(prm[2:5]); l = prm[5]
    for _ in range(5):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        w = rng.uniform(-0.5, 0.5, 3)
        TB = rng.uniform(-1, 2, 3)
        d = oracle.f(MARS6, prm, np.concatenate([[1.5], np.zeros(6), q, w]), TB)
        np.testing.assert_allclose(d[7:11], 0.5 * quat_mul(q, np.concatenate([[0.0], w])), atol=1e-15)
        wd = np.linalg.solve(J, np.cross([-l, 0, 0], TB) - np.cross(w, J @ w))
        np.testing.assert_allclose(d[11:14], wd, atol=1e-13)


def test_mars6_free_fall_and_upright_burn_closed_forms():
    prm = mars6_params()
    x = np.concatenate([[1.5, 2.0, 0.3, -0.2, -0.5, 0.1, 0.0], [1, 0, 0, 0], [0, 0, 0]])
    xt = rollout(MARS6, prm, 0.1, x, np.zeros(3), 10)
    np.testing.assert_allclose(xt[1:4], x[1:4] + x[4:7] + 0.5 * np.array([-prm[1], 0, 0]), atol=1e-13)
    np.testing.assert_allclose(xt[[0] + list(range(7, 14))], x[[0] + list(range(7, 14))], atol=0)
    # upright burn along the body (= world) x axis: the 3-DOF rocket equation
    p3 = mars_params().copy(); p3[0], p3[1] = prm[1], prm[0]
    T = np.array([2.2, 0, 0])
    x3 = np.concatenate([x[1:7], [x[0]]])
    a = rollout(MARS6, prm, 0.05, x, T, 20)
    b = rollout(MARS, p3, 0.05, x3, T, 20)
    np.testing.assert_allclose(a[1:7], b[0:6], atol=1e-14)
    np.testing.assert_allclose(a[0], b[6], atol=1e-15)
