"""Failure detection without a GPU fault: an allocation failure injected on the
host (UCN_FAULT_ALLOC) at every allocation of the two create calls returns
UCN_ENOMEM and leaves no device memory behind; an instance seeded with NaN data
ends UCN_ENUMERIC while every other instance of its launch gives the clean
run's bits; a time budget that has already run out ends every independent
instance UCN_ETIMEOUT after one SCP iteration, and the kernel returns."""
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_10711_gb300 import serving, ucn  # noqa: E402

KEYS = ["defect", "cost", "merit", "primal_res", "dual_res", "tr_radius", "step", "scp_iters", "accepted",
        "accept_mask", "status"]


def free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def fault_sweep(make, close, limit=400):
    """Create with the n-th allocation failing, n = 1, 2, ... until a create
    succeeds; every failure must be an injected ENOMEM.  Returns the number of
    allocations the create makes."""
    n = 1
    try:
        while n <= limit:
            os.environ["UCN_FAULT_ALLOC"] = str(n)
            try:
                h = make()
            except ucn.UcnError as e:
                assert e.status == ucn.UCN_ENOMEM and "injected" in str(e), (n, e)
                n += 1
                continue
            close(h)
            return n - 1
    finally:
        os.environ.pop("UCN_FAULT_ALLOC", None)
    raise AssertionError("no create succeeded")


def test_injected_allocation_failures_return_enomem_and_leak_nothing():
    # a batch big enough that one leaked array would show (the exported ADMM state
    # alone is ~14 MB), created first once to load the library and its kernels
    prob = W.mars_batch(256, seed=3, N=100, settings=dict(scp_iters=3))
    desc, keep = ucn.make_desc(prob, ucn.UCN_PREC_FP32_REFINE)
    ref = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE)
    xr, ur = ref.scp_solve()
    xr, ur, sr = xr.cpu().numpy(), ur.cpu().numpy(), ref.stats_host()
    ref.close()
    ucn.ucn_problem_destroy(ucn.ucn_problem_create(desc))
    before = free_bytes()
    for _ in range(2):
        count = fault_sweep(lambda: ucn.ucn_problem_create(desc), ucn.ucn_problem_destroy)
        assert count >= 20
    after = free_bytes()
    assert abs(after - before) <= 4 << 20, (before, after)
    # the library still works and gives the same bits
    s = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE)
    x, u = s.scp_solve()
    np.testing.assert_array_equal(x.cpu().numpy(), xr)
    np.testing.assert_array_equal(u.cpu().numpy(), ur)
    s.close()


def test_injected_allocation_failures_of_the_server_leak_nothing():
    settings = dict(W.mars_batch(1).settings)

    def make():
        return serving.Server(2, ucn.UCN_PREC_FP32_REFINE, max_slots=256, max_horizon=100, lanes=4, settings=settings)

    make().close()
    before = free_bytes()
    for _ in range(2):
        count = fault_sweep(make, lambda s: s.close())
        assert count >= 30
    after = free_bytes()
    assert abs(after - before) <= 4 << 20, (before, after)
    srv = make()
    p = W.mars_batch(1, seed=11, N=60)
    rc, t = srv.submit(p); srv.pump()
    for _ in range(1000000):
        rc, res = srv.poll(t, horizon=60)
        if rc == ucn.UCN_OK:
            break
    assert rc == ucn.UCN_OK and res["stats"]["status"] == ucn.UCN_OK
    srv.close()


def solve(prob, precision, **kw):
    s = ucn.Solver(prob, precision=precision, **kw)
    x, u = s.scp_solve()
    out = x.cpu().numpy(), u.cpu().numpy(), s.stats_host()
    s.close()
    return out


def nan_cases():
    return [
        ("mars", ucn.UCN_PREC_FP32_REFINE, lambda: W.mars_batch(16, seed=5, N=60, settings=dict(scp_iters=30))),
        ("mars", ucn.UCN_PREC_FP64, lambda: W.mars_batch(16, seed=5, N=60, settings=dict(scp_iters=30))),
        ("quad", ucn.UCN_PREC_FP32_REFINE,
         lambda: W.quad_box(16, seed=6, N_range=(20, 40), obs_range=(2, 6), settings=dict(scp_iters=8, admm_iters=60))),
        ("quad", ucn.UCN_PREC_FP64,
         lambda: W.quad_box(16, seed=6, N_range=(20, 40), obs_range=(2, 6), settings=dict(scp_iters=8, admm_iters=60))),
    ]


@pytest.mark.parametrize("name,precision,make", nan_cases(), ids=["mars32", "mars64", "quad32", "quad64"])
def test_nan_instance_ends_enumeric_and_leaves_the_others_unchanged(name, precision, make):
    prob = make()
    xc, uc, sc = solve(prob, precision)
    bad = 5
    seeded = make()
    seeded.xinit = seeded.xinit.copy()
    seeded.xinit[bad, 0] = np.nan
    xs, us, ss = solve(seeded, precision)
    assert ss["status"][bad] == ucn.UCN_ENUMERIC
    for b in range(prob.batch):
        if b == bad:
            continue
        xo, uo, N = prob.xoff[b], prob.uoff[b], int(prob.N[b])
        np.testing.assert_array_equal(xs[xo:xo + N + 1], xc[xo:xo + N + 1])
        np.testing.assert_array_equal(us[uo:uo + N], uc[uo:uo + N])
        for k in KEYS:
            assert ss[k][b] == sc[k][b] or (np.isnan(ss[k][b]) and np.isnan(sc[k][b])), (b, k)


@pytest.mark.parametrize("name,precision,make", nan_cases(), ids=["mars32", "mars64", "quad32", "quad64"])
def test_spent_time_budget_ends_every_independent_instance_etimeout(name, precision, make):
    prob = make()
    x, u, st = solve(prob, precision, timeout_s=1e-9)
    assert (st["status"] == ucn.UCN_ETIMEOUT).all()
    assert (st["scp_iters"] == 1).all()
    # the returned trajectory is the nominal after that one iteration: finite, and
    # starting at the initial state
    assert np.isfinite(x).all() and np.isfinite(u).all()
    np.testing.assert_array_equal(x[prob.xoff], prob.xinit)
