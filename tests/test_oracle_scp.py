"""Pins of the oracle's SCP loop (Sec. III-A) on the two workload models.

* a nominal produced by an RK4 rollout has zero dynamics defect, so the
  merit of the first nominal equals its cost, computed here from the
  problem data;
* the nominal carried to the next iteration is the candidate when it is
  accepted and the old nominal otherwise (bookkeeping of the acceptance test);
* converged solves reach the defect level the method is measured at
  (max |RK4(x_i,u_i) - x_{i+1}|_inf <= 1e-5), satisfy the boundary
  conditions of Eq. (1c) and the control sets exactly, and keep clear of the
  obstacles / inside the thrust and glide-slope sets.
"""
import math

import numpy as np

import oracle
import workloads as W


def instance(prob, x, u, b):
    xo, uo, N = prob.xoff[b], prob.uoff[b], int(prob.N[b])
    return x[xo:xo + N + 1], u[uo:uo + N]


def cost(prob, b, x, u):
    """phi(x_N) + sum l(x_i, u_i) of Eq. (1a), from the problem data."""
    N = int(prob.N[b])
    ex = x - prob.xref[b]; eu = u - prob.uref[b]
    c = 0.5 * np.sum(prob.Qd[b] * ex[:N] ** 2) + 0.5 * np.sum(prob.Rd[b] * eu ** 2)
    c += 0.5 * np.sum(prob.QNd[b] * ex[N] ** 2) + prob.qN[b] @ x[N]
    return c


def max_defect(prob, b, x, u):
    N = int(prob.N[b])
    return max(np.abs(oracle.rk4(prob.model, prob.params[b], prob.dt[b], x[i], u[i]) - x[i + 1]).max()
               for i in range(N))


def test_rollout_nominal_has_zero_defect_and_merit_equals_cost():
    prob = W.quad_path(1, seed=3, settings=dict(scp_iters=1, admm_iters=5))
    N = int(prob.N[0])
    u = prob.uguess.copy()
    u[:, 1] += 0.05 * np.sin(np.arange(N))
    x = np.zeros((N + 1, 12)); x[0] = prob.xinit[0]
    for i in range(N):
        x[i + 1] = oracle.rk4(1, prob.params[0], prob.dt[0], x[i], u[i])
    _, _, _, log = oracle.scp_solve(prob, xguess=x, uguess=u, log=True)
    assert max_defect(prob, 0, x, u) == 0.0
    assert abs(log[0, 0, 2] - cost(prob, 0, x, u)) < 1e-9 * max(1.0, abs(cost(prob, 0, x, u)))


def test_nominal_bookkeeping_follows_accept_flags():
    prob = W.quad_path(1, seed=0)
    _, _, st, log = oracle.scp_solve(prob, log=True)
    K = int(prob.settings["scp_iters"])
    for k in range(K - 1):
        expect = log[0, k, 3] if log[0, k, 0] == 1 else log[0, k, 2]
        assert abs(log[0, k + 1, 2] - expect) <= 1e-9 * max(1.0, abs(expect))
    assert st[0, 8] == np.sum(log[0, :, 0])


def test_quadrotor_converges_and_respects_sets():
    # with rho = 10 the solves reach the defect level (rho = 1 needs far more iterations)
    prob = W.quad_path(4, seed=0, settings=dict(rho_eq=10.0, rho_dyn=10.0, rho_geo=10.0, scp_iters=40,
                                                stop=1, step_tol=1.0))
    x, u, st, _ = oracle.scp_solve(prob)
    for b in range(4):
        xb, ub = instance(prob, x, u, b)
        assert st[b, 0] <= 1e-5 and st[b, 10] == 0
        assert abs(max_defect(prob, b, xb, ub) - st[b, 0]) < 1e-15
        np.testing.assert_array_equal(xb[0], prob.xinit[b])                   # x_0 = x_init
        np.testing.assert_array_equal(xb[-1][:6], prob.xtarget[b][:6])        # S x_N = x_target
        assert ub.min() >= prob.ulo[b].min() and ub.max() <= prob.uhi[b].max()  # control box
        for j in range(prob.nobs[b]):
            dist = np.linalg.norm(xb[:, :3] - prob.obs_c[b, j], axis=1)
            assert dist.min() >= prob.obs_r[b, j] - 1e-4


def test_mars_converges_and_respects_sets():
    prob = W.mars_batch(3, seed=1)
    x, u, st, _ = oracle.scp_solve(prob)
    tmin, tmax, tang = prob.sets[0, :3]
    for b in range(3):
        xb, ub = instance(prob, x, u, b)
        assert st[b, 0] <= 1e-5 and st[b, 10] == 0
        assert st[b, 7] < prob.settings["scp_iters"]                          # stopped by the test
        np.testing.assert_array_equal(xb[0], prob.xinit[b])
        np.testing.assert_array_equal(xb[-1][:6], 0.0)
        Tn = np.linalg.norm(ub, axis=1)
        assert Tn.max() <= tmax + 1e-4 and Tn.min() >= tmin - 1e-4             # thrust annulus
        horiz = np.hypot(xb[:, 1], xb[:, 2])
        assert np.all(horiz <= tang * xb[:, 0] + 1e-4)                        # glide slope
        assert xb[:, 6].min() >= prob.xlo[b, 6] and np.all(np.diff(xb[:, 6]) <= 1e-5)   # mass only falls


def test_quaternion_quadrotor_converges_and_respects_sets():
    # the 13-state study task with a longer schedule (rho 10 -> 1e3 over 80 iterations)
    prob = W.quat_study(3, rho0=10.0, rho_final=1e3, scp_iters=80, admm_iters=250,
                        settings=dict(stop=1, step_tol=1.0))
    x, u, st, _ = oracle.scp_solve(prob)
    for b in range(3):
        xb, ub = instance(prob, x, u, b)
        assert st[b, 0] <= 1e-5 and st[b, 10] == 0
        assert abs(max_defect(prob, b, xb, ub) - st[b, 0]) < 1e-15
        np.testing.assert_array_equal(xb[0], prob.xinit[b])
        np.testing.assert_array_equal(xb[-1][:6], prob.xtarget[b][:6])        # position, zero velocity
        assert np.all(ub >= prob.ulo[b] - 1e-9) and np.all(ub <= prob.uhi[b] + 1e-9)
        for j in range(prob.nobs[b]):
            dist = np.linalg.norm(xb[:, :3] - prob.obs_c[b, j], axis=1)
            assert dist.min() >= prob.obs_r[b, j] - 1e-3
        # the quaternion stays a rotation to the accuracy the defect allows
        assert np.abs(np.linalg.norm(xb[:, 6:10], axis=1) - 1.0).max() < 0.05


def test_mars6_converges_and_respects_sets():
    prob = W.mars6_batch(3, seed=7)
    x, u, st, _ = oracle.scp_solve(prob)
    tmin, tmax, tglide, tgimbal, rtilt, wmax = prob.sets[0, :6]
    for b in range(3):
        xb, ub = instance(prob, x, u, b)
        assert st[b, 0] <= 1e-5 and st[b, 10] == 0
        np.testing.assert_array_equal(xb[0], prob.xinit[b])
        np.testing.assert_array_equal(xb[-1][1:7], prob.xtarget[b][1:7])          # touchdown
        np.testing.assert_array_equal(xb[-1][9:11], 0.0)                          # upright
        Tn = np.linalg.norm(ub, axis=1)
        assert Tn.max() <= tmax + 1e-4 and Tn.min() >= tmin - 1e-4                 # thrust annulus
        assert np.all(np.hypot(ub[:, 1], ub[:, 2]) <= tgimbal * ub[:, 0] + 1e-4)    # gimbal
        assert np.all(np.hypot(xb[:, 2], xb[:, 3]) <= tglide * xb[:, 1] + 1e-4)     # glide slope
        assert np.all(np.hypot(xb[:, 9], xb[:, 10]) <= rtilt + 1e-4)               # tilt
        assert np.all(np.linalg.norm(xb[:, 11:14], axis=1) <= wmax + 1e-4)          # body rate
        assert xb[:, 0].min() >= 0.75 and np.all(np.diff(xb[:, 0]) <= 1e-5)         # mass


def test_fixed_count_solve_runs_every_iteration():
    prob = W.quad_path(1, seed=0)
    _, _, st, log = oracle.scp_solve(prob, log=True)
    assert st[0, 7] == prob.settings["scp_iters"]
    assert np.all(np.isfinite(log[0, :, 2]))


def test_exact_iteration_count_solve_agrees_with_the_stop_test_and_the_cap():
    # run to each instance's own stopping iteration: the stop-test solve, bit for bit;
    # run to the cap: the solve without a stop test, bit for bit
    for prob in (W.mars_batch(3, seed=1, N=30), W.scenario_mpc(2, 3, seed=3, N=10, n_obs=2,
                                                               settings=dict(scp_iters=12, admm_iters=30))):
        x, u, st, _ = oracle.scp_solve(prob)
        xs, us, ss = oracle.scp_solve_iters(prob, st[:, 7].astype(int))
        np.testing.assert_array_equal(xs, x)
        np.testing.assert_array_equal(us, u)
        np.testing.assert_array_equal(ss[:, 7], st[:, 7])
        K = int(prob.settings["scp_iters"])
        nostop = prob.subset(np.arange(prob.batch))
        nostop.settings["stop"] = 0
        x0, u0, s0, _ = oracle.scp_solve(nostop)
        xk, uk, sk = oracle.scp_solve_iters(prob, np.full(prob.batch, K))
        np.testing.assert_array_equal(xk, x0)
        np.testing.assert_array_equal(uk, u0)
        assert (sk[:, 7] == K).all()


def test_trajectory_defects_are_the_rk4_defects():
    prob = W.mars_batch(3, seed=2, N=25)
    x, u, st, _ = oracle.scp_solve(prob)
    d = oracle.traj_defects(prob, x, u)
    np.testing.assert_array_equal(d, st[:, 0])
    for b in range(prob.batch):
        xb, ub = instance(prob, x, u, b)
        ref = max(np.abs(oracle.rk4(prob.model, prob.params[b], prob.dt[b], xb[i], ub[i]) - xb[i + 1]).max()
                  for i in range(int(prob.N[b])))
        assert d[b] == ref


def test_batch_comparison_reruns_instances_that_stopped_elsewhere():
    prob = W.mars_batch(3, seed=1, N=30)
    ref = oracle.scp_solve(prob)[:3]
    it = ref[2][:, 7].astype(int)
    r = oracle.compare_batch(prob, ref[0], ref[1], it, ref, 1e-4)
    assert r["summary"]["max_rel_err"] == 0.0 and r["summary"]["scp_iters_mismatch"] == 0
    # a solve that ran one more iteration on instance 1 is compared after that many
    it2 = it.copy(); it2[1] += 1
    xs, us, _ = oracle.scp_solve_iters(prob, it2)
    r = oracle.compare_batch(prob, xs, us, it2, ref, 1e-4)
    assert list(r["mismatch"]) == [1] and r["summary"]["max_rel_err"] == 0.0
    # ... whereas against the stop-test solve it differs
    assert oracle.rel_err(xs, ref[0]) > 0.0


def cold_state(prob):
    """The flat ADMM state of the cold start: x = x-hat = z = the guess, u = u-hat,
    zero duals and mirrors (the mirrors are re-projected at the first iteration)."""
    mb = oracle.maxblk(prob)
    parts = []
    for b in range(prob.batch):
        N = int(prob.N[b])
        xb, ub = instance(prob, prob.xguess, prob.uguess, b)
        st = np.zeros(oracle.state_size(N, prob.nx, prob.nu, mb))
        S = oracle.unpack_state(st, N, prob.nx, prob.nu, mb)
        S["x"][:] = xb; S["xh"][:] = xb; S["z"][1:] = xb[1:]; S["u"][:] = ub; S["uh"][:] = ub
        parts.append(st)
    return np.concatenate(parts)


def test_warm_start_from_the_cold_state_is_the_cold_solve():
    # the state plumbing: starting from the state the cold start builds gives the cold
    # solve bit for bit (variables in the flat layout's order, mirrors re-projected); a
    # warm start keeps the schedule's final penalties, so a scheduled problem is compared
    # with its cold solve at those penalties throughout
    for prob in (W.mars_batch(2, seed=3, N=30), W.quad_path(1, seed=1, N=15, settings=dict(scp_iters=5, admm_iters=60))):
        const = prob.subset(np.arange(prob.batch))
        st_ = const.settings
        if st_.get("rho_final", 0.0) > 0:
            f = st_["rho_final"] / st_["rho_geo"]
            st_.update(rho_eq=st_["rho_eq"] * f, rho_dyn=st_["rho_dyn"] * f, rho_geo=st_["rho_geo"] * f, rho_final=0.0)
        x, u, st, _ = oracle.scp_solve(const)
        xw, uw, sw = oracle.scp_solve_warm(prob, cold_state(prob))
        np.testing.assert_array_equal(xw, x)
        np.testing.assert_array_equal(uw, u)
        np.testing.assert_array_equal(sw[:, 7], st[:, 7])
