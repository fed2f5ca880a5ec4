"""Serving on the GPU: a request's result is the same alone and in the mix,
admission respects slots and the HBM budget, warm starts from kept device
trajectories, and a mixed Poisson stream completes with oracle-checked results."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_10711_gb300 import serving, ucn  # noqa: E402

QSET = dict(W.DEFAULT_SETTINGS, rho_eq=10.0, rho_dyn=10.0, rho_geo=10.0, scp_iters=8, admm_iters=60, stop=0)


def quad_req(seed, N, nobs):
    return W.quad_box(1, seed=seed, N_range=(N, N), obs_range=(nobs, nobs), settings=dict(QSET))


def wait(srv, ticket, N, tries=200000):
    for _ in range(tries):
        rc, res = srv.poll(ticket, horizon=N)
        if rc == ucn.UCN_OK:
            return res
    raise AssertionError("request did not finish")


@pytest.mark.parametrize("prec", [ucn.UCN_PREC_FP32_REFINE, ucn.UCN_PREC_FP64])
def test_result_is_the_same_alone_and_in_the_mix(prec):
    srv = serving.Server(1, prec, max_slots=16, max_horizon=60, max_obs=8, lanes=3, settings=QSET)
    target = quad_req(7, 40, 6)
    rc, t = srv.submit(target)
    assert rc == ucn.UCN_OK
    srv.pump()
    alone = wait(srv, t, 40)
    others = [quad_req(100 + k, 20 + 3 * k, 2 + k % 6) for k in range(10)]
    tickets = []
    for k, p in enumerate(others):
        rc, tk = srv.submit(p); assert rc == ucn.UCN_OK; tickets.append((tk, int(p.N[0])))
        if k == 4:
            rc, t2 = srv.submit(target); assert rc == ucn.UCN_OK
    rc, launched = srv.pump()
    assert launched == 11
    mixed = wait(srv, t2, 40)
    for tk, N in tickets:
        wait(srv, tk, N)
    np.testing.assert_array_equal(mixed["x"], alone["x"])
    np.testing.assert_array_equal(mixed["u"], alone["u"])
    assert mixed["stats"]["scp_iters"] == alone["stats"]["scp_iters"]
    xr, ur, sr, _ = oracle.scp_solve(target)
    tol = 1e-9 if prec == ucn.UCN_PREC_FP64 else 1e-4
    assert np.abs(alone["x"] - xr).max() <= tol * max(1.0, np.abs(xr).max())
    srv.close()


def test_admission_by_slots_and_hbm_budget():
    srv = serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=2, max_horizon=40, max_obs=4, lanes=1, settings=QSET)
    assert srv.free_slots() == 2
    assert srv.submit(quad_req(1, 30, 3))[0] == ucn.UCN_OK
    assert srv.submit(quad_req(2, 30, 3))[0] == ucn.UCN_OK
    assert srv.submit(quad_req(3, 30, 3))[0] == ucn.UCN_EBUSY
    assert "slot" in ucn.ucn_last_error()
    srv.close()
    small = serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=8, max_horizon=40, max_obs=4, lanes=1,
                           settings=QSET, hbm_budget_bytes=40000.0)
    assert small.submit(quad_req(4, 10, 2))[0] == ucn.UCN_OK            # a short request fits
    rc, _ = small.submit(quad_req(5, 40, 4))                             # a long one does not
    assert rc == ucn.UCN_EBUSY and "HBM budget" in ucn.ucn_last_error()
    small.close()


def test_warm_start_from_a_kept_trajectory():
    srv = serving.Server(2, ucn.UCN_PREC_FP32_REFINE, max_slots=4, max_horizon=60, lanes=2,
                         settings=dict(W.mars_batch(1).settings))
    p = W.mars_batch(1, seed=11, N=60)
    rc, t = srv.submit(p); srv.pump()
    first = wait(srv, t, 60)
    assert first["stats"]["defect"] <= 1e-5
    rc, t2 = srv.submit(p, warm_ticket=t); assert rc == ucn.UCN_OK
    srv.pump()
    second = wait(srv, t2, 60)
    # started from a converged trajectory: it stops sooner, stays converged and keeps
    # the fuel cost (the optimum is a flat face of an LP-like problem, so the
    # trajectory itself may slide along it)
    assert second["stats"]["defect"] <= 1e-5
    assert second["stats"]["scp_iters"] < first["stats"]["scp_iters"]
    assert abs(second["stats"]["cost"] - first["stats"]["cost"]) < 1e-3
    np.testing.assert_array_equal(second["x"][0], p.xinit[0])
    with pytest.raises(ucn.UcnError):
        srv.submit(p, warm_ticket=987654)
    srv.close()


def test_mixed_stream_completes_and_matches_the_oracle():
    stream = W.serving_stream(24, rate=4000.0, seed=9)
    qs = stream[0][1].settings if stream[0][1].model == 1 else W.quad_box(1).settings
    ms = dict(W.mars_batch(1).settings, rho_final=1e7, scp_iters=80, admm_iters=60)   # Mars N up to 200
    servers = {1: serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=32, max_horizon=120, max_obs=30, lanes=3, settings=qs),
               2: serving.Server(2, ucn.UCN_PREC_FP32_REFINE, max_slots=32, max_horizon=200, lanes=3, settings=ms)}
    out = serving.run_stream(stream, servers)
    assert out["completed"] == 24
    assert out["pass_rate"] >= 0.9
    # two requests of the stream through the server, checked against the oracle
    for arr, p in stream[:2]:
        srv = servers[p.model]
        rc, t = srv.submit(p); srv.pump()
        res = wait(srv, t, int(p.N[0]))
        q = p.subset(np.arange(1))
        q.settings = dict(qs if p.model == 1 else ms)        # the server's schedule, not the request's
        xr, ur, sr, _ = oracle.scp_solve(q)
        if sr[0, 0] <= 1e-5 and res["stats"]["defect"] <= 1e-5:
            assert np.abs(res["x"] - xr).max() <= 1e-3 * max(1.0, np.abs(xr).max())
    for s in servers.values():
        s.close()


@pytest.mark.parametrize("kind", ["quat13", "mars14"])
def test_paper_model_variants_serve_like_the_oracle(kind):
    # the 13-state quaternion quadrotor and the 6-DOF Mars lander through the slot pool,
    # two requests at once, each checked against the oracle's solve of the same problem
    if kind == "quat13":
        probs = [W.quat_study(1, seed=s, scp_iters=6, admm_iters=40) for s in (5, 6)]
        srv = serving.Server(3, ucn.UCN_PREC_FP64, max_slots=4, max_horizon=60, max_obs=3, lanes=2,
                             settings=probs[0].settings)
    else:
        probs = [W.mars6_batch(1, seed=s, settings=dict(scp_iters=6, admm_iters=40, stop=0)) for s in (7, 8)]
        srv = serving.Server(4, ucn.UCN_PREC_FP64, max_slots=4, max_horizon=40, lanes=2, settings=probs[0].settings)
    tickets = []
    for p in probs:
        rc, t = srv.submit(p); assert rc == ucn.UCN_OK
        tickets.append(t)
    srv.pump()
    for p, t in zip(probs, tickets):
        N = int(p.N[0])
        res = wait(srv, t, N)
        xr, ur, sr, _ = oracle.scp_solve(p)
        assert np.abs(res["x"] - xr).max() <= 1e-9 * max(1.0, np.abs(xr).max())
        assert np.abs(res["u"] - ur).max() <= 1e-9 * max(1.0, np.abs(ur).max())
        assert res["stats"]["scp_iters"] == int(sr[0, 7])
    srv.close()
