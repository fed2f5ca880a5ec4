"""The device-resident request loop (ucn_serve_loop_start): a persistent kernel
whose CTAs claim requests as they are submitted and solve each with the fused
solve's body.  Results match the oracle at the stated tolerances and the pump
launches' results; a request is the same bits alone and in the mix; requests
that arrive while others run are claimed by free CTAs and overlap with them on
the device; warm starts read kept results; an idle loop ends by itself and the
next request relaunches it; stop serves what is queued first."""
import time

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


def wait(srv, ticket, N, limit_s=60.0):
    t0 = time.monotonic()
    while time.monotonic() - t0 < limit_s:
        rc, res = srv.poll(ticket, horizon=N)
        if rc == ucn.UCN_OK:
            return res
    raise AssertionError("request %d did not finish within %.0f s" % (ticket, limit_s))


def rel(a, b):
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.mark.parametrize("prec", [ucn.UCN_PREC_FP32_REFINE, ucn.UCN_PREC_FP64])
def test_loop_results_match_the_oracle_and_the_pump_launches(prec):
    tol = 1e-9 if prec == ucn.UCN_PREC_FP64 else 1e-4
    reqs = [quad_req(600 + k, 16 + 6 * k, 1 + k % 7) for k in range(8)]
    pump = serving.Server(1, prec, max_slots=8, max_horizon=60, max_obs=8, lanes=2, settings=QSET)
    tp = [pump.submit(p)[1] for p in reqs]
    pump.pump()
    rp = [wait(pump, t, int(p.N[0])) for t, p in zip(tp, reqs)]
    pump.close()
    srv = serving.Server(1, prec, max_slots=8, max_horizon=60, max_obs=8, lanes=2, settings=QSET)
    srv.loop_start(idle_s=5.0)
    tl = []
    for p in reqs:
        rc, t = srv.submit(p)
        assert rc == ucn.UCN_OK
        tl.append(t)
    rl = [wait(srv, t, int(p.N[0])) for t, p in zip(tl, reqs)]
    srv.loop_stop()
    assert srv.loop_launches() == 1
    srv.close()
    for p, a, b in zip(reqs, rl, rp):
        xr, ur, sr, _ = oracle.scp_solve(p)
        assert rel(a["x"], xr) <= tol and rel(a["u"], ur) <= tol
        assert rel(a["x"], b["x"]) <= tol and rel(a["u"], b["u"]) <= tol
        assert a["stats"]["status"] == b["stats"]["status"]
        if prec == ucn.UCN_PREC_FP64:
            assert a["stats"]["scp_iters"] == b["stats"]["scp_iters"] == int(sr[0, 7])


def test_mid_flight_requests_overlap_and_give_their_solo_bits():
    # Mars FP32 (the one-thread-per-node body): a target solved alone through the
    # loop, then again while a first group is on the GPU, with more requests after
    # it; the target starts on the device before the first group has ended and its
    # result is the same bits as alone; every result against the oracle at 1e-4
    st = dict(W.mars_batch(1).settings)
    srv = serving.Server(2, ucn.UCN_PREC_FP32_REFINE, max_slots=32, max_horizon=100, lanes=1, settings=st)
    srv.loop_start(idle_s=5.0)
    target = W.mars_batch(1, seed=21, N=100)
    rc, t = srv.submit(target)
    alone = wait(srv, t, 100)
    first = [W.mars_batch(1, seed=300 + k, N=100) for k in range(12)]
    tk_first = [srv.submit(p)[1] for p in first]
    rc, t2 = srv.submit(target)
    assert rc == ucn.UCN_OK
    later = [W.mars_batch(1, seed=400 + k, N=60 + 10 * k) for k in range(4)]
    tk_later = [srv.submit(p)[1] for p in later]
    mixed = wait(srv, t2, 100)
    firsts = [wait(srv, tk, 100) for tk in tk_first]
    lates = [wait(srv, tk, int(p.N[0])) for tk, p in zip(tk_later, later)]
    srv.loop_stop()
    srv.close()
    assert int(mixed["stats"]["t_start_ns"]) < max(int(r["stats"]["t_end_ns"]) for r in firsts)
    np.testing.assert_array_equal(mixed["x"], alone["x"])
    np.testing.assert_array_equal(mixed["u"], alone["u"])
    assert mixed["stats"]["scp_iters"] == alone["stats"]["scp_iters"]
    for p, r in [(target, alone)] + list(zip(first, firsts)) + list(zip(later, lates)):
        q = p.subset(np.arange(1))
        ref = oracle.scp_solve(q)[:3]
        c = oracle.compare_batch(q, r["x"], r["u"], np.array([r["stats"]["scp_iters"]]), ref, 1e-4)
        assert c["summary"]["n_over_tol"] == 0, c["summary"]
        if ref[2][0, 0] <= 1e-5:
            assert c["fp64_defect"][0] <= 1e-5 and r["stats"]["defect"] <= 1e-5


def test_warm_start_through_the_loop_matches_the_oracle():
    # FP64: the second request names the first, delivered one; it starts from that
    # result's trajectory and ADMM state and matches the oracle started the same way
    st = dict(W.mars_batch(1).settings, scp_iters=60)
    srv = serving.Server(2, ucn.UCN_PREC_FP64, max_slots=2, max_horizon=40, lanes=1, settings=st)
    srv.loop_start(idle_s=5.0)
    p1 = W.mars_batch(1, seed=12, N=40)
    rc, t1 = srv.submit(p1)
    r1 = wait(srv, t1, 40)
    s = ucn.Solver(p1, precision=ucn.UCN_PREC_FP64)
    x1, _ = s.scp_solve()
    state = s.state_export().cpu().numpy()
    torch.cuda.synchronize()
    s.close()
    assert rel(r1["x"], x1.cpu().numpy()) <= 1e-12
    q = p1.subset(np.arange(1))
    q.xinit = q.xinit.copy()
    q.xinit[:, 0:3] += np.array([0.004, 0.002, -0.003])
    rc, t2 = srv.submit(q, warm_ticket=t1)
    assert rc == ucn.UCN_OK
    r2 = wait(srv, t2, 40)
    srv.loop_stop()
    srv.close()
    xr, ur, sr = oracle.scp_solve_warm(q, state, xguess=r1["x"], uguess=r1["u"])
    assert r2["stats"]["scp_iters"] == int(sr[0, 7])
    assert rel(r2["x"], xr) <= 1e-9 and rel(r2["u"], ur) <= 1e-9


def test_idle_loop_ends_and_the_next_request_relaunches_it():
    srv = serving.Server(1, ucn.UCN_PREC_FP32_REFINE, max_slots=4, max_horizon=40, max_obs=4, lanes=1, settings=QSET)
    p = quad_req(31, 30, 3)
    rc, t = srv.submit(p)                 # admitted before the loop starts: published at start
    srv.loop_start(idle_s=0.2)
    r0 = wait(srv, t, 30)
    time.sleep(0.8)                       # every CTA has found nothing for 0.2 s and ended
    rc, t1 = srv.submit(p)                # the submit sees the ended launch and relaunches
    assert rc == ucn.UCN_OK
    r1 = wait(srv, t1, 30)
    assert srv.loop_launches() == 2
    np.testing.assert_array_equal(r1["x"], r0["x"])
    # stop serves every published request before the kernel ends
    tickets = [srv.submit(quad_req(40 + k, 20 + 5 * k, k))[1] for k in range(4)]
    srv.loop_stop()
    for k, tk in enumerate(tickets):
        rc, res = srv.poll(tk, horizon=20 + 5 * k)
        assert rc == ucn.UCN_OK
    # back to pump launches (the lane kernel there may be its other register class):
    # the same request within the FP32 tolerance
    rc, t2 = srv.submit(p)
    srv.pump()
    r2 = wait(srv, t2, 30)
    assert rel(r2["x"], r0["x"]) <= 1e-4
    srv.close()


@pytest.mark.parametrize("kind", ["quat13", "mars14"])
def test_paper_model_variants_through_the_loop_match_the_oracle(kind):
    # the 13-state quaternion quadrotor and the 6-DOF Mars lander through the loop
    # (one thread per node), two requests in flight, each against the oracle in FP64
    if kind == "quat13":
        probs = [W.quat_study(1, seed=s, scp_iters=6, admm_iters=40) for s in (5, 6)]
        srv = serving.Server(3, ucn.UCN_PREC_FP64, max_slots=4, max_horizon=60, max_obs=3, lanes=1,
                             settings=probs[0].settings)
    else:
        probs = [W.mars6_batch(1, seed=s, settings=dict(scp_iters=6, admm_iters=40, stop=0)) for s in (7, 8)]
        srv = serving.Server(4, ucn.UCN_PREC_FP64, max_slots=4, max_horizon=40, lanes=1, settings=probs[0].settings)
    srv.loop_start(idle_s=5.0)
    tickets = []
    for p in probs:
        rc, t = srv.submit(p)
        assert rc == ucn.UCN_OK
        tickets.append(t)
    res = [wait(srv, t, int(p.N[0])) for p, t in zip(probs, tickets)]
    srv.loop_stop()
    srv.close()
    for p, r in zip(probs, res):
        xr, ur, sr, _ = oracle.scp_solve(p)
        assert rel(r["x"], xr) <= 1e-9 and rel(r["u"], ur) <= 1e-9
        assert r["stats"]["scp_iters"] == int(sr[0, 7])


def test_a_second_loop_start_is_rejected():
    srv = serving.Server(1, ucn.UCN_PREC_FP64, max_slots=2, max_horizon=40, max_obs=4, lanes=1, settings=QSET)
    assert srv.loop_capacity() >= torch.cuda.get_device_properties(0).multi_processor_count
    srv.loop_start(idle_s=0.5)
    with pytest.raises(ucn.UcnError) as e:
        srv.loop_start()
    assert e.value.status == ucn.UCN_EINVAL
    srv.loop_stop()
    srv.close()
