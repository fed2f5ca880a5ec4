"""Pins of the oracle's scenario groups (robust MPC, Sec. IV-A): the first
control is shared inside a group, K identical scenarios reproduce the
single-instance solve exactly, and a group of one is an independent instance."""
import numpy as np

import oracle
import workloads as W


def test_group_of_identical_scenarios_equals_single_solve():
    single = W.quad_box(1, seed=6, N_range=(20, 20), obs_range=(4, 4), settings=dict(scp_iters=5, admm_iters=80, stop=0))
    xs, us, ss, _ = oracle.scp_solve(single)
    grp = single.subset([0, 0, 0])
    grp.settings["group"] = 3
    xg, ug, sg, _ = oracle.scp_solve(grp)
    for k in range(3):
        np.testing.assert_allclose(xg[k * 21:(k + 1) * 21], xs, rtol=0, atol=1e-13)
        np.testing.assert_allclose(ug[k * 20:(k + 1) * 20], us, rtol=0, atol=1e-13)
    assert (sg[:, 8] == ss[0, 8]).all()          # same accept decisions


def test_scenarios_share_the_first_control():
    prob = W.scenario_mpc(P=2, K=4, N=20, n_obs=3, settings=dict(scp_iters=6, admm_iters=80, stop=0))
    x, u, st, log = oracle.scp_solve(prob, log=True)
    for p in range(2):
        u0 = np.array([u[prob.uoff[p * 4 + s]] for s in range(4)])
        np.testing.assert_array_equal(u0, np.repeat(u0[:1], 4, axis=0))
        # the scenarios' dynamics differ: their later controls do not coincide
        u5 = np.array([u[prob.uoff[p * 4 + s] + 5] for s in range(4)])
        assert np.abs(u5 - u5[0]).max() > 1e-6
        # one acceptance decision per group
        assert (log[p * 4:(p + 1) * 4, :, 0] == log[p * 4, :, 0]).all()


def test_group_of_one_is_an_independent_instance():
    prob = W.quad_box(3, seed=8, N_range=(15, 25), obs_range=(2, 5), settings=dict(scp_iters=4, admm_iters=50, stop=0))
    x1, u1, s1, _ = oracle.scp_solve(prob)
    prob.settings["group"] = 1
    x2, u2, s2, _ = oracle.scp_solve(prob)
    np.testing.assert_array_equal(x1, x2)
