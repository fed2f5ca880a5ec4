"""ucn_scp_solve_noalloc -- the solve for callers that cannot allocate device
memory (real-time loops, applications whose pool owns the GPU) -- against the
allocating entry point ucn_scp_solve, on the same inputs, twice in a row (the
two calls share the library's static scratch array).

Tolerances are those of the parity tests: FP64 1e-9, FP32 1e-4 (normwise,
floor 1).  This file is collected last so that a failure here stops a -x run
only after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_10711_gb300 import ucn  # noqa: E402

FIELDS = [("dt", "dt"), ("model_params", "params"), ("Q_diag", "Qd"), ("x_ref", "xref"), ("R_diag", "Rd"),
          ("u_ref", "uref"), ("QN_diag", "QNd"), ("qN", "qN"), ("x_lo", "xlo"), ("x_hi", "xhi"), ("u_lo", "ulo"),
          ("u_hi", "uhi"), ("x_init", "xinit"), ("x_target", "xtarget"), ("obs_c", "obs_c"), ("obs_r", "obs_r"),
          ("sets", "sets")]


def device_desc(prob, precision):
    """A descriptor whose arrays (all but the host horizon) live on the GPU."""
    desc, keep = ucn.make_desc(prob, precision)
    held = [keep]
    for cname, attr in FIELDS:
        a = np.ascontiguousarray(getattr(prob, attr), dtype=np.float64)
        t = torch.as_tensor(a if a.size else np.zeros(1), device="cuda")
        held.append(t)
        setattr(desc, cname, C.cast(C.c_void_p(t.data_ptr()), C.POINTER(C.c_double)))
    tm = torch.as_tensor(np.ascontiguousarray(prob.tmask, dtype=np.uint8), device="cuda")
    no = torch.as_tensor(np.ascontiguousarray(prob.nobs, dtype=np.int32), device="cuda")
    held += [tm, no]
    desc.term_mask = C.cast(C.c_void_p(tm.data_ptr()), C.POINTER(C.c_ubyte))
    desc.n_obs = C.cast(C.c_void_p(no.data_ptr()), C.POINTER(C.c_int))
    return desc, held


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


@pytest.mark.parametrize("name,precision,tol", [
    ("quad", ucn.UCN_PREC_FP64, 1e-9),
    ("mars", ucn.UCN_PREC_FP32_REFINE, 1e-4),
])
def test_noalloc_matches_allocating_entry_point_twice(name, precision, tol):
    prob = (W.quad_path(2, seed=0, settings=dict(scp_iters=6, admm_iters=80)) if name == "quad"
            else W.mars_batch(8, seed=1, N=60, settings=dict(scp_iters=40)))
    ref = ucn.Solver(prob, precision=precision)
    xr, ur = ref.scp_solve()
    torch.cuda.synchronize()
    xr, ur, sr = xr.cpu().numpy(), ur.cpu().numpy(), ref.stats_host()
    ref.close()
    desc, held = device_desc(prob, precision)
    x0 = torch.as_tensor(prob.xguess, device="cuda"); u0 = torch.as_tensor(prob.uguess, device="cuda")
    for call in range(2):
        xo = torch.full_like(x0, np.nan); uo = torch.full_like(u0, np.nan)
        stats = torch.zeros(prob.batch * 128, dtype=torch.uint8, device="cuda")
        status = torch.full((prob.batch,), -1, dtype=torch.int32, device="cuda")
        ucn.ucn_scp_solve_noalloc(desc, x0, u0, xo, uo, stats, status)
        torch.cuda.synchronize()
        st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=ucn.STATS_DTYPE)
        assert rel_err(xo.cpu().numpy(), xr) <= tol, (call, rel_err(xo.cpu().numpy(), xr))
        assert rel_err(uo.cpu().numpy(), ur) <= tol, call
        np.testing.assert_array_equal(st["scp_iters"], sr["scp_iters"])
        np.testing.assert_array_equal(status.cpu().numpy(), sr["status"])
        assert rel_err(st["defect"], sr["defect"]) <= tol


def test_noalloc_rejects_batches_beyond_its_scratch():
    prob = W.mars_batch(1300, seed=1, N=100)     # ~72 MB of state > 64 MiB
    desc, held = device_desc(prob, ucn.UCN_PREC_FP32_REFINE)
    x0 = torch.as_tensor(prob.xguess, device="cuda"); u0 = torch.as_tensor(prob.uguess, device="cuda")
    stats = torch.zeros(prob.batch * 128, dtype=torch.uint8, device="cuda")
    status = torch.zeros(prob.batch, dtype=torch.int32, device="cuda")
    with pytest.raises(ucn.UcnError) as ei:
        ucn.ucn_scp_solve_noalloc(desc, x0, u0, x0.clone(), u0.clone(), stats, status)
    assert ei.value.status == ucn.UCN_EINVAL and "scratch" in str(ei.value)


def noalloc_solve(prob, precision, desc=None, held=None):
    if desc is None:
        desc, held = device_desc(prob, precision)
    x0 = torch.as_tensor(prob.xguess, device="cuda"); u0 = torch.as_tensor(prob.uguess, device="cuda")
    xo = torch.full_like(x0, np.nan); uo = torch.full_like(u0, np.nan)
    stats = torch.zeros(prob.batch * 128, dtype=torch.uint8, device="cuda")
    status = torch.full((prob.batch,), -1, dtype=torch.int32, device="cuda")
    ucn.ucn_scp_solve_noalloc(desc, x0, u0, xo, uo, stats, status)
    torch.cuda.synchronize()
    return xo.cpu().numpy(), uo.cpu().numpy(), np.frombuffer(stats.cpu().numpy().tobytes(), dtype=ucn.STATS_DTYPE)


def test_noalloc_uneven_batch_over_several_table_chunks():
    # 1000 uneven horizons: the horizons reach the device in two by-value chunks and the
    # offsets come from the device-side scan with several instances per thread
    prob = W.quad_box(1000, seed=8, N_range=(3, 24), obs_range=(0, 3), settings=dict(scp_iters=2, admm_iters=15, stop=0))
    ref = ucn.Solver(prob, precision=ucn.UCN_PREC_FP64)
    xr, ur = ref.scp_solve()
    torch.cuda.synchronize()
    xr, ur, sr = xr.cpu().numpy(), ur.cpu().numpy(), ref.stats_host()
    ref.close()
    xo, uo, st = noalloc_solve(prob, ucn.UCN_PREC_FP64)
    assert rel_err(xo, xr) <= 1e-9 and rel_err(uo, ur) <= 1e-9
    np.testing.assert_array_equal(st["scp_iters"], sr["scp_iters"])


def test_noalloc_clamps_obstacle_counts_beyond_max_obs():
    # a device n_obs above max_obs (which only the host-side create can reject) is read as
    # max_obs: the solve ends and matches the same problem with n_obs = max_obs
    prob = W.quad_path(2, seed=0, n_obs=5, settings=dict(scp_iters=4, admm_iters=40))
    x5, u5, s5 = noalloc_solve(prob, ucn.UCN_PREC_FP64)
    desc, held = device_desc(prob, ucn.UCN_PREC_FP64)
    bad = torch.tensor([9, 64], dtype=torch.int32, device="cuda")
    held.append(bad)
    desc.n_obs = C.cast(C.c_void_p(bad.data_ptr()), C.POINTER(C.c_int))
    x9, u9, s9 = noalloc_solve(prob, ucn.UCN_PREC_FP64, desc, held)
    np.testing.assert_array_equal(x9, x5)
    np.testing.assert_array_equal(u9, u5)
    np.testing.assert_array_equal(s9["status"], s5["status"])
