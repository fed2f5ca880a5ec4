"""Serving on the GPU: a request's result is the same alone and in the mix
(also when it arrives while another launch runs), admission respects slots and
the HBM budget, warm starts from kept device trajectories and ADMM states
(against the oracle started from the same state), and a mixed Poisson stream
completes with every result oracle-checked."""
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


def test_warm_start_from_a_kept_result():
    srv = serving.Server(2, ucn.UCN_PREC_FP32_REFINE, max_slots=4, max_horizon=60, lanes=2,
                         settings=dict(W.mars_batch(1).settings))
    p = W.mars_batch(1, seed=11, N=60)
    rc, t = srv.submit(p); srv.pump()
    first = wait(srv, t, 60)
    assert first["stats"]["defect"] <= 1e-5
    rc, t2 = srv.submit(p, warm_ticket=t); assert rc == ucn.UCN_OK
    srv.pump()
    second = wait(srv, t2, 60)
    # started from a converged trajectory and its ADMM state: it stops sooner, stays
    # converged and keeps the fuel cost (the optimum is a flat face of an LP-like
    # problem, so the trajectory itself may slide along it)
    assert second["stats"]["defect"] <= 1e-5
    assert second["stats"]["scp_iters"] < first["stats"]["scp_iters"]
    assert abs(second["stats"]["cost"] - first["stats"]["cost"]) < 1e-3
    np.testing.assert_array_equal(second["x"][0], p.xinit[0])
    with pytest.raises(ucn.UcnError):
        srv.submit(p, warm_ticket=987654)
    srv.close()


def moved(prob, dr):
    q = prob.subset(np.arange(prob.batch))
    q.xinit = q.xinit.copy()
    q.xinit[:, 0:3] += dr
    return q


def test_warm_start_from_kept_state_matches_the_oracle():
    # a request that names a finished one starts from its kept trajectory AND ADMM
    # state; in FP64 it matches the oracle started from the same state and guess (the
    # kept state of the first request, taken from the same solve through a problem)
    st = dict(W.mars_batch(1).settings, scp_iters=60)
    srv = serving.Server(2, ucn.UCN_PREC_FP64, max_slots=2, max_horizon=40, lanes=1, settings=st)
    p1 = W.mars_batch(1, seed=12, N=40)
    rc, t1 = srv.submit(p1); srv.pump()
    r1 = wait(srv, t1, 40)
    s = ucn.Solver(p1, precision=ucn.UCN_PREC_FP64)
    x1, _ = s.scp_solve()
    state = s.state_export().cpu().numpy()
    torch.cuda.synchronize()
    s.close()
    assert np.abs(x1.cpu().numpy() - r1["x"]).max() <= 1e-12 * max(1.0, np.abs(r1["x"]).max())
    p2 = moved(p1, np.array([0.004, 0.002, -0.003]))
    rc, t2 = srv.submit(p2, warm_ticket=t1); assert rc == ucn.UCN_OK
    srv.pump()
    r2 = wait(srv, t2, 40)
    srv.close()
    xr, ur, sr = oracle.scp_solve_warm(p2, state, xguess=r1["x"], uguess=r1["u"])
    assert r2["stats"]["scp_iters"] == int(sr[0, 7])
    assert np.abs(r2["x"] - xr).max() <= 1e-9 * max(1.0, np.abs(xr).max())
    assert np.abs(r2["u"] - ur).max() <= 1e-9 * max(1.0, np.abs(ur).max())


def test_request_admitted_mid_flight_overlaps_and_matches_its_solo_run():
    # continuous batching: a first group runs on one lane; the target arrives while it
    # is on the GPU, is admitted and launched on another lane, and more requests come
    # after it; the launches overlap on the device and the target's result is the same
    # bits as when it runs alone
    for prec in (ucn.UCN_PREC_FP32_REFINE, ucn.UCN_PREC_FP64):
        srv = serving.Server(1, prec, max_slots=32, max_horizon=60, max_obs=8, lanes=4, settings=QSET)
        target = quad_req(7, 40, 6)
        rc, t = srv.submit(target); srv.pump()
        alone = wait(srv, t, 40)
        first = [quad_req(200 + k, 60, 8) for k in range(12)]
        tk_first = []
        for p in first:
            rc, tk = srv.submit(p); assert rc == ucn.UCN_OK; tk_first.append(tk)
        rc, n1 = srv.pump(); assert n1 == 12
        rc, t2 = srv.submit(target); assert rc == ucn.UCN_OK   # while the first launch runs
        rc, n2 = srv.pump(); assert n2 == 1
        later = [quad_req(300 + k, 30, 4) for k in range(5)]
        tk_later = []
        for p in later:
            rc, tk = srv.submit(p); assert rc == ucn.UCN_OK; tk_later.append(tk)
        rc, n3 = srv.pump(); assert n3 == 5
        mixed = wait(srv, t2, 40)
        firsts = [wait(srv, tk, 60) for tk in tk_first]
        for tk in tk_later:
            wait(srv, tk, 30)
        srv.close()
        # the target's launch ran while the first launch was still running
        f_end = max(int(r["stats"]["t_end_ns"]) for r in firsts)
        assert int(mixed["stats"]["t_start_ns"]) < f_end
        np.testing.assert_array_equal(mixed["x"], alone["x"])
        np.testing.assert_array_equal(mixed["u"], alone["u"])
        assert mixed["stats"]["scp_iters"] == alone["stats"]["scp_iters"]


def test_slots_reused_while_launches_run_give_the_solo_results():
    # four slots, three lanes, 16 requests: every slot is reused several times while
    # other launches still run (a freed slot waits for its launch to end before it
    # takes a new request); poll_any hands out each result once, bit-identical to the
    # request solved alone
    reqs = [quad_req(500 + k, 12 + 7 * (k % 5), k % 4) for k in range(16)]
    solo = []
    one = serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=1, max_horizon=60, max_obs=8, lanes=1, settings=QSET)
    for p in reqs:
        rc, t = one.submit(p); one.pump()
        solo.append(wait(one, t, int(p.N[0])))
    one.close()
    srv = serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=4, max_horizon=60, max_obs=8, lanes=3, settings=QSET)
    pending, got, which = list(range(16)), {}, {}
    for _ in range(2000000):
        while pending and srv.free_slots() > 0:
            k = pending.pop(0)
            rc, t = srv.submit(reqs[k]); assert rc == ucn.UCN_OK
            which[t] = k
        srv.pump()
        rc, t, res = srv.poll_any(trajectories=True)
        if rc == ucn.UCN_OK:
            assert t not in got
            got[t] = res
        if len(got) == 16:
            break
    assert len(got) == 16 and srv.poll_any()[0] == ucn.UCN_EBUSY
    srv.close()
    for t, res in got.items():
        ref = solo[which[t]]
        np.testing.assert_array_equal(res["x"], ref["x"])
        np.testing.assert_array_equal(res["u"], ref["u"])
        assert res["stats"]["scp_iters"] == ref["stats"]["scp_iters"]


def test_mixed_stream_completes_and_every_result_matches_the_oracle():
    stream = W.serving_stream(24, rate=4000.0, seed=9)
    qs = W.quad_box(1).settings
    ms = dict(W.mars_batch(1).settings, rho_final=1e7, scp_iters=80, admm_iters=60)   # Mars N up to 200
    servers = {1: serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=32, max_horizon=120, max_obs=30, lanes=3, settings=qs),
               2: serving.Server(2, ucn.UCN_PREC_FP32_REFINE, max_slots=32, max_horizon=200, lanes=3, settings=ms)}
    out = serving.run_stream(stream, servers)
    assert out["completed"] == 24
    # every request of the stream through the servers again, each result against the
    # oracle's solve of it on the server's schedule: 1e-4 after the same SCP iteration
    # count, and the FP64 defect gate wherever the oracle reaches it
    tickets = []
    for arr, p in stream:
        rc, t = servers[p.model].submit(p); assert rc == ucn.UCN_OK
        tickets.append(t)
    for srv in servers.values():
        srv.pump()
    for (arr, p), t in zip(stream, tickets):
        res = wait(servers[p.model], t, int(p.N[0]))
        q = p.subset(np.arange(1))
        q.settings = dict(qs if p.model == 1 else ms)        # the server's schedule, not the request's
        ref = oracle.scp_solve(q)[:3]
        r = oracle.compare_batch(q, res["x"], res["u"], np.array([res["stats"]["scp_iters"]]), ref, 1e-4)
        assert r["summary"]["n_over_tol"] == 0, (p.model, int(p.N[0]), r["summary"])
        if ref[2][0, 0] <= 1e-5:
            assert r["fp64_defect"][0] <= 1e-5 and res["stats"]["defect"] <= 1e-5
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
