"""Pins of the oracle's SCP acceptance test and trust-region update.

The paper leaves the trust-region logic out (Sec. III-A); the solver adopts
this reading: merit J = cost + w_d * sum_i |RK4(x_i, u_i) - x_{i+1}|_1, its
linear model L with A_i x_i + B_i u_i + d_i in place of RK4, ratio =
(J(nominal) - J(candidate)) / (J(nominal) - L(candidate)); accept when the
model decrease is <= 1e-12 or the ratio is > 0; the radius halves below 0.25,
doubles (capped at tr_max) above 0.75, and is floored at tr_min.  Scenario
groups take the same decision on the sums of J and L over their scenarios.

Each case runs ONE SCP iteration of the oracle and recomputes J(nominal),
J(candidate) and L(candidate) here from their definitions -- the cost
l = 1/2 |x - x_ref|^2_Q + 1/2 |u - u_ref|^2_R, phi = 1/2 |x_N - x_ref|^2_QN
+ qN^T x_N, the RK4 step and the linearisation of Eq. (2b) (both pinned in
test_oracle_models.py against closed forms and complex-step derivatives) and
the candidate of the ADMM of Sec. III-B (pinned in test_oracle_admm.py) --
then checks the logged values, the decision and the new radius against the
rule written out below.  The cases are chosen so that every branch of the
rule is taken at least once.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def cost(prob, b, x, u):
    N = int(prob.N[b])
    c = 0.0
    for i in range(N):
        e = x[i] - prob.xref[b]
        c += 0.5 * np.sum(prob.Qd[b] * e * e)
        e = u[i] - prob.uref[b]
        c += 0.5 * np.sum(prob.Rd[b] * e * e)
    e = x[N] - prob.xref[b]
    return c + 0.5 * np.sum(prob.QNd[b] * e * e) + float(prob.qN[b] @ x[N])


def linearisation(prob, b, x, u):
    N = int(prob.N[b])
    A = np.zeros((N, prob.nx, prob.nx)); B = np.zeros((N, prob.nx, prob.nu)); d = np.zeros((N, prob.nx))
    for i in range(N):
        A[i], B[i], d[i], _ = oracle.linearize(prob.model, prob.params[b], prob.dt[b], x[i], u[i])
    return A, B, d


def merits(prob, b, xbar, ubar, xc, uc, w_d):
    """(J(nominal), J(candidate), L(candidate), rounding scale of L)."""
    N = int(prob.N[b])
    A, B, d = linearisation(prob, b, xbar, ubar)
    f = lambda x, u: oracle.rk4(prob.model, prob.params[b], prob.dt[b], x, u)
    nl_n = sum(np.abs(f(xbar[i], ubar[i]) - xbar[i + 1]).sum() for i in range(N))
    nl_c = sum(np.abs(f(xc[i], uc[i]) - xc[i + 1]).sum() for i in range(N))
    lin = [A[i] @ xc[i] + B[i] @ uc[i] + d[i] - xc[i + 1] for i in range(N)]
    # the linear defects cancel large terms (d_i = RK4 - A xbar - B ubar): their
    # rounding is relative to the magnitude of those terms, not of the result
    mag = sum((np.abs(d[i]) + np.abs(A[i]) @ np.abs(xc[i]) + np.abs(B[i]) @ np.abs(uc[i])
               + np.abs(xc[i + 1])).sum() for i in range(N))
    cc = cost(prob, b, xc, uc)
    return (cost(prob, b, xbar, ubar) + w_d * nl_n, cc + w_d * nl_c,
            cc + w_d * sum(np.abs(v).sum() for v in lin), w_d * mag + abs(cc))


def rule(Jn, Jc, Lc, radius, tr_min, tr_max):
    """The acceptance reading written out: (branch, accept, new radius, ratio)."""
    den, num = Jn - Lc, Jn - Jc
    if den <= 1e-12:
        return "no model decrease", True, max(radius, tr_min), np.nan
    ratio = num / den
    r = radius
    if ratio < 0.25:
        r = 0.5 * radius
    elif ratio > 0.75:
        r = min(2.0 * radius, tr_max)
    branch = ("reject" if ratio <= 0 else "accept, shrink" if ratio < 0.25 else
              "accept, keep" if ratio <= 0.75 else "accept, grow")
    if r < tr_min:
        branch += ", floor"
    elif ratio > 0.75 and 2.0 * radius > tr_max:
        branch += ", cap"
    return branch, ratio > 0, max(r, tr_min), ratio


def rollout_problem(seed, ang, rate, rad, w_d, tr_min=1e-6, tr_max=10.0, admm=400, rho=10.0, N=12):
    """One quadrotor whose nominal is an exact RK4 rollout from a tilted,
    spinning start (zero defect), free terminal state: the candidate of a large
    trust region then trades cost decrease against nonlinear defect."""
    p = W.quad_path(1, seed=0, N=N, settings=dict(scp_iters=1, admm_iters=admm, tr_init=rad, tr_min=tr_min,
                                                 tr_max=tr_max, rho_eq=rho, rho_dyn=rho, rho_geo=rho, w_d=w_d))
    p.tmask[:] = 0
    rng = np.random.default_rng(seed)
    x0 = p.xinit[0].copy()
    x0[6:9] = ang * rng.standard_normal(3)
    x0[9:12] = rate * rng.standard_normal(3)
    p.xinit[0] = x0
    u = p.uguess + 0.5 * rng.standard_normal(p.uguess.shape)
    x = np.zeros_like(p.xguess)
    x[0] = x0
    for i in range(N):
        x[i + 1] = oracle.rk4(p.model, p.params[0], p.dt[0], x[i], u[i])
    p.xguess[:] = x
    p.uguess[:] = u
    return p


# (name, builder arguments, branch expected)
CASES = [
    ("no model decrease", dict(seed=1, ang=0.5, rate=2.0, rad=0.5, w_d=1e3), "no model decrease"),
    ("reject", dict(seed=1, ang=1.2, rate=10.0, rad=10.0, w_d=60.0), "reject"),
    ("shrink", dict(seed=1, ang=1.2, rate=10.0, rad=3.0, w_d=60.0), "accept, shrink"),
    ("keep", dict(seed=1, ang=1.2, rate=10.0, rad=3.0, w_d=30.0), "accept, keep"),
    ("grow", dict(seed=1, ang=1.2, rate=10.0, rad=1.0, w_d=30.0), "accept, grow"),
    ("grow to the cap", dict(seed=1, ang=1.2, rate=10.0, rad=1.0, w_d=30.0, tr_max=1.5), "accept, grow, cap"),
    ("shrink to the floor", dict(seed=1, ang=1.2, rate=10.0, rad=3.0, w_d=60.0, tr_min=2.0), "accept, shrink, floor"),
    ("reject to the floor", dict(seed=1, ang=1.2, rate=10.0, rad=10.0, w_d=60.0, tr_min=7.0), "reject, floor"),
]


@pytest.mark.parametrize("name,kw,branch", CASES, ids=[c[0] for c in CASES])
def test_single_instance_acceptance_rule(name, kw, branch):
    prob = rollout_problem(**kw)
    s = prob.settings
    N = int(prob.N[0])
    xbar, ubar = prob.xguess.copy(), prob.uguess.copy()
    # the candidate: one ADMM call on the QP of Eq. (2) at the nominal, from a cold start
    A, B, d = linearisation(prob, 0, xbar, ubar)
    st, _, rc = oracle.problem_admm(prob, 0, xbar, ubar, A, B, d, s["tr_init"], s["admm_iters"])
    assert rc == 0
    S = oracle.unpack_state(st, N, prob.nx, prob.nu, oracle.maxblk(prob))
    xc, uc = S["xh"], S["uh"]
    Jn, Jc, Lc, mag = merits(prob, 0, xbar, ubar, xc, uc, s["w_d"])
    got_branch, acc, radius, ratio = rule(Jn, Jc, Lc, s["tr_init"], s["tr_min"], s["tr_max"])
    assert got_branch == branch

    xo, uo, so, lg = oracle.scp_solve(prob, log=True)
    L = lg[0, 0]
    assert abs(L[2] - Jn) <= 1e-12 * abs(Jn)
    assert abs(L[3] - Jc) <= 1e-12 * abs(Jc)
    assert abs(L[4] - Lc) <= 1e-12 * mag
    if np.isnan(ratio):
        assert np.isnan(L[1])
    else:
        assert abs(L[1] - ratio) <= 1e-9 * max(1.0, abs(ratio))
    assert bool(L[0]) == acc
    assert L[6] == radius and so[0, 5] == radius
    assert int(so[0, 8]) == int(acc) and int(so[0, 9]) == int(acc)
    # accepted: the candidate is the new nominal (returned); rejected: the nominal stays
    np.testing.assert_array_equal(xo, xc if acc else xbar)
    np.testing.assert_array_equal(uo, uc if acc else ubar)


def group_problem(rad, w_d, K=2):
    """Two scenarios (masses 1 and 1.05 kg) of the rollout problem, coupled by
    their first control (Sec. IV-A)."""
    p = rollout_problem(seed=1, ang=1.2, rate=10.0, rad=rad, w_d=w_d)
    g = p.subset(np.zeros(K, dtype=int))
    g.params[1:, 0] = 1.05
    g.settings["group"] = K
    return g


@pytest.mark.parametrize("rad,w_d,branch", [(3.0, 60.0, "accept, shrink"), (10.0, 60.0, "reject"),
                                            (1.0, 30.0, "accept, grow"), (3.0, 30.0, "accept, keep")])
def test_group_acceptance_rule(rad, w_d, branch):
    g = group_problem(rad, w_d)
    # the group's candidates do not depend on w_d (it enters the merit only): a
    # run with w_d = 1, whose candidate is accepted, returns them
    gc = group_problem(rad, 1.0)
    xc_all, uc_all, sc, lc = oracle.scp_solve(gc, log=True)
    assert (lc[:, 0, 0] == 1).all()
    Jn = Jc = Lc = mag = 0.0
    for b in range(g.batch):
        xo_, uo_, N = g.xoff[b], g.uoff[b], int(g.N[b])
        jn, jc, lc_, m = merits(g, b, g.xguess[xo_:xo_ + N + 1], g.uguess[uo_:uo_ + N],
                                xc_all[xo_:xo_ + N + 1], uc_all[uo_:uo_ + N], w_d)
        Jn += jn; Jc += jc; Lc += lc_; mag += m
    got_branch, acc, radius, ratio = rule(Jn, Jc, Lc, rad, g.settings["tr_min"], g.settings["tr_max"])
    assert got_branch == branch
    xo, uo, so, lg = oracle.scp_solve(g, log=True)
    for b in range(g.batch):
        L = lg[b, 0]
        assert abs(L[2] - Jn) <= 1e-12 * abs(Jn)
        assert abs(L[3] - Jc) <= 1e-12 * abs(Jc)
        assert abs(L[4] - Lc) <= 1e-12 * mag
        assert abs(L[1] - ratio) <= 1e-9 * max(1.0, abs(ratio))
        assert bool(L[0]) == acc and L[6] == radius
    np.testing.assert_array_equal(xo, xc_all if acc else g.xguess)
    np.testing.assert_array_equal(uo, uc_all if acc else g.uguess)
