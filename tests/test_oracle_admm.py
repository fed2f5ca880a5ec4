"""Pins of the oracle's consensus ADMM (Sec. III-B, Eq. (3)-(8)) and projections.

The ADMM is tied to: a dense whole-horizon KKT solve and a Riccati recursion
(unconstrained linear-quadratic instances), brute-force active-set
enumeration (tiny box / half-space instances), a multiplier root-find (a
ball-constrained instance), the defining minimisations of each ADMM step
(evaluated on the augmented Lagrangian of Eq. (3) written out here), and the
monotone Lyapunov quantity of two-block ADMM (the convergence remark,
Sec. III-B).
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W

INF = np.inf
HALF, BALL, CONE, NONE = oracle.BLK_HALF, oracle.BLK_BALL, oracle.BLK_CONE, oracle.BLK_NONE


def free_qp(seed, N=4, nx=3, nu=2):
    qp = W.double_integrator(seed=seed, N=N, nx=nx, nu=nu)
    qp.update(xlo=np.full((N + 1, nx), -INF), xhi=np.full((N + 1, nx), INF),
              ulo=np.full((N, nu), -INF), uhi=np.full((N, nu), INF))
    return qp


def dense_kkt(qp, extra_eq=None, active=()):
    """Minimise the QP of Eq. (2) subject to x_0 = x_init, the dynamics and
    optional extra equalities (rows, rhs); returns (z, multipliers)."""
    N, nx, nu = qp["N"], qp["nx"], qp["nu"]
    nv = (N + 1) * nx + N * nu
    xi = lambda i: slice(i * nx, (i + 1) * nx)
    ui = lambda i: slice((N + 1) * nx + i * nu, (N + 1) * nx + (i + 1) * nu)
    H = np.zeros((nv, nv)); c = np.zeros(nv)
    for i in range(N + 1):
        H[xi(i), xi(i)] += qp["Q"][i]; c[xi(i)] += qp["q"][i]
    for i in range(N):
        H[ui(i), ui(i)] += qp["R"][i]; c[ui(i)] += qp["r"][i]
        H[xi(i), ui(i)] += qp["M"][i]; H[ui(i), xi(i)] += qp["M"][i].T
    E = [np.zeros((nx, nv))]; E[0][:, xi(0)] = np.eye(nx); e = [qp["x0"]]
    for i in range(N):
        r = np.zeros((nx, nv)); r[:, xi(i + 1)] = np.eye(nx); r[:, xi(i)] -= qp["A"][i]; r[:, ui(i)] -= qp["B"][i]
        E.append(r); e.append(qp["d"][i])
    if extra_eq is not None:
        E.append(extra_eq[0]); e.append(extra_eq[1])
    E = np.vstack(E); e = np.concatenate(e)
    K = np.block([[H, E.T], [E, np.zeros((E.shape[0], E.shape[0]))]])
    sol = np.linalg.solve(K, np.concatenate([-c, e]))
    return sol[:nv], sol[nv:], (xi, ui, nv)


def riccati(qp):
    """Backward Riccati recursion for the affine LQ problem with cross terms:
    V_i(x) = 1/2 x^T P x + p^T x; u_i = -K x - k; forward rollout from x0."""
    N = qp["N"]
    P = qp["Q"][N].copy(); p = qp["q"][N].copy()
    Ks, ks = [None] * N, [None] * N
    for i in reversed(range(N)):
        A, B, d = qp["A"][i], qp["B"][i], qp["d"][i]
        Qi, Ri, Mi, qi, ri = qp["Q"][i], qp["R"][i], qp["M"][i], qp["q"][i], qp["r"][i]
        Huu = Ri + B.T @ P @ B
        Hux = Mi.T + B.T @ P @ A
        hu = ri + B.T @ (P @ d + p)
        K = np.linalg.solve(Huu, Hux); k = np.linalg.solve(Huu, hu)
        Hxx = Qi + A.T @ P @ A
        hx = qi + A.T @ (P @ d + p)
        P = Hxx - Hux.T @ K
        p = hx - Hux.T @ k
        P = 0.5 * (P + P.T)
        Ks[i], ks[i] = K, k
    x = qp["x0"].copy(); xs = [x]; us = []
    for i in range(N):
        u = -Ks[i] @ x - ks[i]
        x = qp["A"][i] @ x + qp["B"][i] @ u + qp["d"][i]
        us.append(u); xs.append(x)
    return np.array(xs), np.array(us)


def run_admm(qp, iters, rho=(1.0, 1.0, 1.0)):
    st, stats, rc = oracle.admm_qp(qp, iters, rho=rho)
    assert rc == 0
    mb = qp.get("blk_kind", np.zeros((qp["N"] + 1, 0))).shape[1]
    return oracle.unpack_state(st, qp["N"], qp["nx"], qp["nu"], mb), stats


# ------------------------------------------------------------------ LQ pins
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("rho", [(1.0, 1.0, 1.0), (2.0, 0.7, 3.0)])
def test_unconstrained_lq_matches_dense_kkt_and_riccati(seed, rho):
    qp = free_qp(seed)
    S, stats = run_admm(qp, 6000, rho)
    sol, _, (xi, ui, nv) = dense_kkt(qp)
    N, nx, nu = qp["N"], qp["nx"], qp["nu"]
    xd = sol[:(N + 1) * nx].reshape(N + 1, nx); ud = sol[(N + 1) * nx:].reshape(N, nu)
    xr, ur = riccati(qp)
    np.testing.assert_allclose(xd, xr, atol=1e-11)          # the two references agree
    np.testing.assert_allclose(S["x"], xd, atol=1e-10)
    np.testing.assert_allclose(S["u"], ud, atol=1e-10)
    np.testing.assert_allclose(S["xh"], xd, atol=1e-10)      # mirrors agree at the fixed point
    np.testing.assert_allclose(S["z"][1:], xd[1:], atol=1e-10)
    assert stats[0] < 1e-10 and stats[1] < 1e-10


def test_terminal_selection_constraint_matches_dense_kkt():
    qp = free_qp(7, N=5, nx=3, nu=1)
    N, nx = qp["N"], qp["nx"]
    qp["tmask"] = np.array([1, 0, 1], np.uint8)
    qp["xtarget"] = np.array([0.4, 9.0, -0.3])
    S, _ = run_admm(qp, 20000)
    nv = (N + 1) * nx + N * qp["nu"]
    rows = np.zeros((2, nv)); rows[0, N * nx + 0] = 1; rows[1, N * nx + 2] = 1
    sol, _, _ = dense_kkt(qp, extra_eq=(rows, np.array([0.4, -0.3])))
    np.testing.assert_allclose(S["x"].ravel(), sol[:(N + 1) * nx], atol=1e-9)
    assert abs(S["xh"][N, 1] - S["x"][N, 1]) < 1e-9   # the unselected component is free


# ------------------------------------------------------------------ brute force
def add_blocks(qp, mb):
    N, nx, nu = qp["N"], qp["nx"], qp["nu"]
    qp["blk_kind"] = np.full((N + 1, mb), NONE, np.int32)
    qp["blk_G"] = np.zeros((N + 1, mb, 3, nx + nu))
    qp["blk_p"] = np.zeros((N + 1, mb))


def brute_force_qp(qp, ineqs):
    """Enumerate active sets of inequalities g^T v >= b (v the stacked
    variable); the unique point that is feasible with nonnegative multipliers
    is the optimum of the strictly convex QP."""
    best = None
    n = len(ineqs)
    for act in itertools.product([0, 1], repeat=n):
        idx = [k for k in range(n) if act[k]]
        N, nx, nu = qp["N"], qp["nx"], qp["nu"]
        nv = (N + 1) * nx + N * nu
        rows = np.array([ineqs[k][0] for k in idx]).reshape(len(idx), nv)
        rhs = np.array([ineqs[k][1] for k in idx])
        try:
            v, lam, _ = dense_kkt(qp, extra_eq=(rows, rhs))
        except np.linalg.LinAlgError:
            continue
        feas = all(g @ v >= b - 1e-10 for g, b in ineqs)
        mult = lam[lam.size - len(idx):] if idx else np.zeros(0)
        # KKT of min f s.t. g^T v >= b: grad f = sum lam g with lam >= 0; the
        # equality multipliers returned by dense_kkt carry the opposite sign
        if feas and np.all(-mult >= -1e-10):
            assert best is None or np.allclose(best, v, atol=1e-8)
            best = v
    assert best is not None
    return best


@pytest.mark.parametrize("seed", range(3))
def test_box_and_halfspace_instance_matches_active_set_enumeration(seed):
    qp = W.double_integrator(seed=seed + 20, N=2, nx=2, nu=1)
    N, nx, nu = 2, 2, 1
    nv = (N + 1) * nx + N * nu
    qp["q"] = qp["q"] * 4.0; qp["r"] = qp["r"] * 4.0     # push the optimum into the constraints
    qp["x0"] = np.array([0.3, 0.1])                       # a start from which the sets are reachable
    ulo, uhi = -0.3, 0.25
    qp.update(xlo=np.full((N + 1, nx), -INF), xhi=np.full((N + 1, nx), INF),
              ulo=np.full((N, nu), ulo), uhi=np.full((N, nu), uhi))
    qp["xlo"][2, 1] = -0.2                                  # one state bound
    add_blocks(qp, 1)
    nrm = np.array([0.6, 0.8])
    for i in (1, 2):                                        # a half-space on each later state
        qp["blk_kind"][i, 0] = HALF
        qp["blk_G"][i, 0, 0, :nx] = nrm
        qp["blk_p"][i, 0] = 0.05 * i
    ineqs = []
    for i in range(N):
        g = np.zeros(nv); g[(N + 1) * nx + i] = 1; ineqs.append((g, ulo))
        g = np.zeros(nv); g[(N + 1) * nx + i] = -1; ineqs.append((g, -uhi))
    g = np.zeros(nv); g[2 * nx + 1] = 1; ineqs.append((g, -0.2))
    for i in (1, 2):
        g = np.zeros(nv); g[i * nx:i * nx + nx] = nrm; ineqs.append((g, 0.05 * i))
    ref = brute_force_qp(qp, ineqs)
    S, stats = run_admm(qp, 40000)
    got = np.concatenate([S["xh"].ravel(), S["uh"].ravel()])
    np.testing.assert_allclose(got, ref, atol=1e-9)
    np.testing.assert_allclose(np.concatenate([S["x"].ravel(), S["u"].ravel()]), ref, atol=1e-9)


def test_ball_constrained_instance_matches_multiplier_root():
    # one control ball |u_1| <= R: optimum = dense solve with u_1 penalised by
    # (lam/2)|u_1|^2, lam >= 0 the root of |u_1(lam)| = R
    qp = W.double_integrator(seed=5, N=3, nx=2, nu=2)
    N, nx, nu = 3, 2, 2
    qp["r"] = qp["r"] * 6.0
    qp.update(xlo=np.full((N + 1, nx), -INF), xhi=np.full((N + 1, nx), INF),
              ulo=np.full((N, nu), -INF), uhi=np.full((N, nu), INF))
    R = 0.35
    add_blocks(qp, 1)
    qp["blk_kind"][1, 0] = BALL
    qp["blk_G"][1, 0, 0, nx + 0] = 1; qp["blk_G"][1, 0, 1, nx + 1] = 1
    qp["blk_p"][1, 0] = R
    sl = slice((N + 1) * nx + nu, (N + 1) * nx + 2 * nu)

    def solve(lam):
        q2 = dict(qp); q2["R"] = qp["R"].copy(); q2["R"][1] = qp["R"][1] + lam * np.eye(nu)
        v, _, _ = dense_kkt(q2)
        return v

    v0 = solve(0.0)
    assert np.linalg.norm(v0[sl]) > R                       # the ball is active
    lo, hi = 0.0, 1.0
    while np.linalg.norm(solve(hi)[sl]) > R:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.linalg.norm(solve(mid)[sl]) > R: lo = mid
        else: hi = mid
    ref = solve(0.5 * (lo + hi))
    S, _ = run_admm(qp, 30000)
    got = np.concatenate([S["x"].ravel(), S["u"].ravel()])
    np.testing.assert_allclose(got, ref, atol=1e-9)
    np.testing.assert_allclose(S["s"][1, 0, :2], ref[sl], atol=1e-9)


def test_cone_constrained_instance_matches_slsqp():
    from scipy.optimize import minimize
    qp = W.double_integrator(seed=9, N=2, nx=3, nu=1)
    N, nx, nu = 2, 3, 1
    qp["q"] = qp["q"] * 3.0
    qp["x0"] = np.array([1.0, 0.2, -0.1])                  # inside the cone
    qp.update(xlo=np.full((N + 1, nx), -INF), xhi=np.full((N + 1, nx), INF),
              ulo=np.full((N, nu), -INF), uhi=np.full((N, nu), INF))
    tau = 0.5
    add_blocks(qp, 1)
    for i in (1, 2):
        qp["blk_kind"][i, 0] = CONE
        for k in range(3):
            qp["blk_G"][i, 0, k, k] = 1
        qp["blk_p"][i, 0] = tau
    nv = (N + 1) * nx + N * nu
    _, _, (xi, ui, _) = dense_kkt(qp)

    def obj(v):
        f = 0.0
        for i in range(N + 1):
            x = v[xi(i)]; f += 0.5 * x @ qp["Q"][i] @ x + qp["q"][i] @ x
        for i in range(N):
            x, u = v[xi(i)], v[ui(i)]
            f += 0.5 * u @ qp["R"][i] @ u + x @ qp["M"][i] @ u + qp["r"][i] @ u
        return f

    cons = [{"type": "eq", "fun": lambda v: v[xi(0)] - qp["x0"]}]
    for i in range(N):
        cons.append({"type": "eq", "fun": lambda v, i=i: v[xi(i + 1)] - qp["A"][i] @ v[xi(i)] - qp["B"][i] @ v[ui(i)] - qp["d"][i]})
    for i in (1, 2):
        cons.append({"type": "ineq", "fun": lambda v, i=i: tau ** 2 * v[i * nx] ** 2 - v[i * nx + 1] ** 2 - v[i * nx + 2] ** 2})
        cons.append({"type": "ineq", "fun": lambda v, i=i: v[i * nx]})
    S, _ = run_admm(qp, 40000)
    got = np.concatenate([S["x"].ravel(), S["u"].ravel()])
    res = minimize(obj, got + 0.01, constraints=cons, method="SLSQP", options=dict(ftol=1e-15, maxiter=500))
    assert res.success, res.message
    np.testing.assert_allclose(got, res.x, atol=2e-6)
    assert obj(got) <= obj(res.x) + 1e-9
    for i in (1, 2):   # the cone holds at the solution and is active somewhere
        assert np.hypot(*S["x"][i, 1:3]) <= tau * S["x"][i, 0] + 1e-9


# ------------------------------------------------------------------ one iteration = block minimisation
def lagrangian(qp, S, rho):
    """The augmented Lagrangian of Eq. (3), extended by the mirror blocks, written out term by term."""
    re, rd, rg = rho
    N = qp["N"]
    L = 0.0
    for i in range(N + 1):
        x = S["x"][i]
        L += 0.5 * x @ qp["Q"][i] @ x + qp["q"][i] @ x
        L += S["nux"][i] @ (x - S["xh"][i]) + 0.5 * rg * np.sum((x - S["xh"][i]) ** 2)
        if i >= 1:
            L += S["lam"][i] @ (x - S["z"][i]) + 0.5 * re * np.sum((x - S["z"][i]) ** 2)
    for i in range(N):
        x, u = S["x"][i], S["u"][i]
        L += 0.5 * u @ qp["R"][i] @ u + x @ qp["M"][i] @ u + qp["r"][i] @ u
        dd = qp["A"][i] @ x + qp["B"][i] @ u + qp["d"][i]
        L += S["mu"][i + 1] @ (S["z"][i + 1] - dd) + 0.5 * rd * np.sum((S["z"][i + 1] - dd) ** 2)
        L += S["nuu"][i] @ (u - S["uh"][i]) + 0.5 * rg * np.sum((u - S["uh"][i]) ** 2)
    mb = qp["blk_kind"].shape[1]
    for i in range(N + 1):
        xi = np.concatenate([S["x"][i], S["u"][i] if i < N else np.zeros(qp["nu"])])
        for b in range(mb):
            if qp["blk_kind"][i, b] == NONE:
                continue
            dim = 1 if qp["blk_kind"][i, b] == HALF else 3
            y = qp["blk_G"][i, b, :dim] @ xi - S["s"][i, b, :dim]
            L += S["nus"][i, b, :dim] @ y + 0.5 * rg * y @ y
    return L


def num_grad(fun, S, key, h=1e-3):
    g = np.zeros_like(S[key])
    for idx in np.ndindex(S[key].shape):
        Sp = {k: v.copy() for k, v in S.items()}; Sm = {k: v.copy() for k, v in S.items()}
        Sp[key][idx] += h; Sm[key][idx] -= h
        g[idx] = (fun(Sp) - fun(Sm)) / (2 * h)
    return g


def test_one_iteration_is_the_block_minimisation_of_the_lagrangian():
    rng = np.random.default_rng(4)
    N, nx, nu = 3, 3, 2
    qp = W.double_integrator(seed=13, N=N, nx=nx, nu=nu)
    qp.update(xlo=np.full((N + 1, nx), -0.5), xhi=np.full((N + 1, nx), 0.6),
              ulo=np.full((N, nu), -0.4), uhi=np.full((N, nu), 0.3))
    qp["tmask"] = np.array([1, 0, 0], np.uint8); qp["xtarget"] = np.array([0.2, 0, 0])
    add_blocks(qp, 2)
    for i in range(N + 1):
        qp["blk_kind"][i, 0] = HALF
        qp["blk_G"][i, 0, 0, :nx] = [0.6, 0.0, 0.8]; qp["blk_p"][i, 0] = -0.1
        if i < N:
            qp["blk_kind"][i, 1] = BALL
            qp["blk_G"][i, 1, 0, nx] = 1; qp["blk_G"][i, 1, 1, nx + 1] = 1; qp["blk_p"][i, 1] = 0.3
    rho = (1.3, 0.8, 2.1)
    S0 = oracle.unpack_state(rng.normal(size=oracle.state_size(N, nx, nu, 2)), N, nx, nu, 2)
    S0["z"][0] = 0; S0["lam"][0] = 0; S0["mu"][0] = 0
    S0["s"][:, :, :] *= 0.3
    S0["s"][N, 1] = 0; S0["nus"][N, 1] = 0
    S0["s"][:, 0, 1:] = 0; S0["nus"][:, 0, 1:] = 0; S0["s"][:, 1, 2] = 0; S0["nus"][:, 1, 2] = 0
    flat0 = np.concatenate([S0[k].ravel() for k in ("x", "u", "z", "lam", "mu", "xh", "uh", "nux", "nuu", "s", "nus")])
    st1, _, rc = oracle.admm_qp(qp, 1, state=flat0, rho=rho)
    assert rc == 0
    S1 = oracle.unpack_state(st1, N, nx, nu, 2)
    re, rd, rg = rho
    # Step 1: (x, u) minimise L with every other variable at its old value
    mix = {k: S0[k].copy() for k in S0}; mix["x"] = S1["x"].copy(); mix["u"] = S1["u"].copy()
    for key in ("x", "u"):
        assert np.abs(num_grad(lambda S: lagrangian(qp, S, rho), mix, key)).max() < 1e-8
    # Step 2: z minimises L given the new (x, u) and the old duals
    mix2 = {k: S0[k].copy() for k in S0}
    for k in ("x", "u", "z"): mix2[k] = S1[k].copy()
    gz = num_grad(lambda S: lagrangian(qp, S, rho), mix2, "z")
    assert np.abs(gz[1:]).max() < 1e-8
    # Step 3: the mirrors are projections of (primal + dual/rho)
    v = S1["x"] + S0["nux"] / rg
    exp_xh = np.clip(v, qp["xlo"], qp["xhi"])
    exp_xh[0] = qp["x0"]; exp_xh[N, 0] = 0.2
    np.testing.assert_allclose(S1["xh"], exp_xh, atol=1e-14)
    np.testing.assert_allclose(S1["uh"], np.clip(S1["u"] + S0["nuu"] / rg, qp["ulo"], qp["uhi"]), atol=1e-14)
    for i in range(N + 1):
        y = qp["blk_G"][i, 0, 0, :nx] @ S1["x"][i] + S0["nus"][i, 0, 0] / rg
        assert abs(S1["s"][i, 0, 0] - max(y, -0.1)) < 1e-14
        if i < N:
            y = S1["u"][i] + S0["nus"][i, 1, :2] / rg
            nrm = np.linalg.norm(y)
            np.testing.assert_allclose(S1["s"][i, 1, :2], y * min(1, 0.3 / nrm), atol=1e-14)
    # Step 4: dual ascent on each consensus residual
    for i in range(1, N + 1):
        dd = qp["A"][i - 1] @ S1["x"][i - 1] + qp["B"][i - 1] @ S1["u"][i - 1] + qp["d"][i - 1]
        np.testing.assert_allclose(S1["lam"][i], S0["lam"][i] + re * (S1["x"][i] - S1["z"][i]), atol=1e-13)
        np.testing.assert_allclose(S1["mu"][i], S0["mu"][i] + rd * (S1["z"][i] - dd), atol=1e-13)
    np.testing.assert_allclose(S1["nux"], S0["nux"] + rg * (S1["x"] - S1["xh"]), atol=1e-13)
    np.testing.assert_allclose(S1["nuu"], S0["nuu"] + rg * (S1["u"] - S1["uh"]), atol=1e-13)


# ------------------------------------------------------------------ convergence remark
def test_two_block_lyapunov_quantity_is_nonincreasing():
    """He & Yuan (2015): for two-block ADMM the weighted change of the
    second block and the duals, sum rho |B dv|^2 + |dy|^2 / rho, never grows."""
    N, nx, nu = 4, 3, 2
    qp = W.double_integrator(seed=17, N=N, nx=nx, nu=nu)
    qp["x0"] = np.array([0.3, 0.1, 0.0])                   # feasible start (inside boxes and cone)
    qp.update(xlo=np.full((N + 1, nx), -0.4), xhi=np.full((N + 1, nx), 0.5),
              ulo=np.full((N, nu), -0.2), uhi=np.full((N, nu), 0.2))
    add_blocks(qp, 1)
    for i in range(N + 1):
        qp["blk_kind"][i, 0] = CONE
        for k in range(3): qp["blk_G"][i, 0, k, k] = 1
        qp["blk_p"][i, 0] = 2.0
    rho = (1.5, 0.6, 1.1)
    re, rd, rg = rho
    st, _, _ = oracle.admm_qp(qp, 1, rho=rho)
    prev = oracle.unpack_state(st, N, nx, nu, 1)
    vals = []
    for _ in range(300):
        st, _, _ = oracle.admm_qp(qp, 1, state=st, rho=rho)
        cur = oracle.unpack_state(st, N, nx, nu, 1)
        dz = cur["z"][1:] - prev["z"][1:]
        V = (re + rd) * np.sum(dz ** 2) + rg * (np.sum((cur["xh"] - prev["xh"]) ** 2) + np.sum((cur["uh"] - prev["uh"]) ** 2)
                                              + np.sum((cur["s"] - prev["s"]) ** 2))
        V += np.sum((cur["lam"] - prev["lam"]) ** 2) / re + np.sum((cur["mu"] - prev["mu"]) ** 2) / rd
        V += (np.sum((cur["nux"] - prev["nux"]) ** 2) + np.sum((cur["nuu"] - prev["nuu"]) ** 2)
              + np.sum((cur["nus"] - prev["nus"]) ** 2)) / rg
        vals.append(V)
        prev = cur
    vals = np.array(vals)
    assert np.all(vals[1:] <= vals[:-1] * (1 + 1e-9) + 1e-28)
    assert vals[-1] < 1e-6 * vals[0]


# ------------------------------------------------------------------ projections
@pytest.mark.parametrize("kind,p0,dim", [(HALF, 0.3, 1), (BALL, 0.7, 3), (CONE, 0.5, 3), (CONE, 14.3, 3)])
def test_projection_properties(kind, p0, dim):
    rng = np.random.default_rng(kind + 10)
    P = lambda y: oracle.project(kind, p0, y)

    def member(y):
        if kind == HALF: return y[0] >= p0 - 1e-12
        if kind == BALL: return np.linalg.norm(y) <= p0 + 1e-12
        return np.hypot(y[1], y[2]) <= p0 * y[0] + 1e-12

    for _ in range(200):
        a, b = rng.normal(size=dim) * 2, rng.normal(size=dim) * 2
        pa, pb = P(a), P(b)
        assert member(pa)
        np.testing.assert_allclose(P(pa), pa, atol=1e-13)                     # idempotent
        assert np.linalg.norm(pa - pb) <= np.linalg.norm(a - b) + 1e-12        # non-expansive
        c = P(rng.normal(size=dim) * 3)                                        # any member of the set
        assert (a - pa) @ (c - pa) <= 1e-10                                    # variational inequality
        if member(a):
            np.testing.assert_allclose(pa, a, atol=1e-15)


def test_cone_moreau_decomposition():
    # y = P_K(y) + P_Ko(y) with P_K(y) . P_Ko(y) = 0; the polar of the cone of
    # half-angle atan(tau) is the cone around -t of half-angle atan(1/tau)
    rng = np.random.default_rng(3)
    for tau in (0.5, 1.0, 14.3):
        for _ in range(200):
            y = rng.normal(size=3) * 2
            pk = oracle.project(CONE, tau, y)
            ypol = np.array([-y[0], y[1], y[2]])
            pko = oracle.project(CONE, 1.0 / tau, ypol)
            pko = np.array([-pko[0], pko[1], pko[2]])
            np.testing.assert_allclose(pk + pko, y, atol=1e-12)
            assert abs(pk @ pko) < 1e-11


def test_ball_is_vector_scaling():
    y = np.array([3.0, 4.0, 0.0])
    np.testing.assert_allclose(oracle.project(BALL, 2.0, y), [1.2, 1.6, 0.0], atol=1e-15)
    np.testing.assert_allclose(oracle.project(BALL, 6.0, y), y, atol=0)
