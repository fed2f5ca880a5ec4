"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (normwise, floor 1):  |gpu - oracle|_max <= tol * max(1, |oracle|_max)
  * FP64 plain path:          tol = 1e-9
  * FP32 path with refinement: tol = 1e-4 after the same number of SCP
    iterations, and the FP64 defect of the returned trajectory <= 1e-5 where
    the oracle reaches it.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_10711_gb300 import ucn  # noqa: E402

TOL64, TOL32 = 1e-9, 1e-4


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max())) if b.size else 0.0


def t(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def perturbed_nominal(prob, seed=0, scale=0.05):
    rng = np.random.default_rng(seed)
    x = prob.xguess + scale * rng.standard_normal(prob.xguess.shape)
    u = prob.uguess + scale * rng.standard_normal(prob.uguess.shape)
    for b in range(prob.batch):
        x[prob.xoff[b]] = prob.xinit[b]
    return x, u


def oracle_linearize(prob, x, u):
    nx, nu = prob.nx, prob.nu
    A = np.zeros((prob.total_u, nx, nx)); B = np.zeros((prob.total_u, nx, nu)); d = np.zeros((prob.total_u, nx))
    for b in range(prob.batch):
        for i in range(int(prob.N[b])):
            g = prob.uoff[b] + i
            A[g], B[g], d[g], _ = oracle.linearize(prob.model, prob.params[b], prob.dt[b], x[prob.xoff[b] + i], u[g])
    return A, B, d


PROBLEMS = {
    "quad_path": lambda: W.quad_path(1, seed=0),
    "quad_uneven": lambda: W.quad_box(3, seed=5, N_range=(5, 17), obs_range=(2, 6)),
    "mars": lambda: W.mars_batch(3, seed=1, N=40),
    "quat": lambda: W.quat_study(2, seed=5, N=30, tf=3.6),
    "mars6": lambda: W.mars6_batch(2, seed=7, N=20, tf=3.4),
}


# ------------------------------------------------------------------ linearisation (Eq. (2b))
@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("prec,tol", [(ucn.UCN_PREC_FP64, 1e-12), (ucn.UCN_PREC_FP32_REFINE, 2e-5)])
def test_linearize_matches_oracle(name, prec, tol):
    prob = PROBLEMS[name]()
    x, u = perturbed_nominal(prob)
    s = ucn.Solver(prob, precision=prec)
    A, B, d = s.linearize(t(x), t(u))
    torch.cuda.synchronize()
    Ar, Br, dr = oracle_linearize(prob, x, u)
    assert rel_err(A.cpu().numpy(), Ar) <= tol
    assert rel_err(B.cpu().numpy(), Br) <= tol
    # d = RK4 - A x - B u is evaluated in FP64 with the path's own A, B
    Ag, Bg = A.cpu().numpy(), B.cpu().numpy()
    xs = np.concatenate([x[prob.xoff[b]:prob.xoff[b] + int(prob.N[b])] for b in range(prob.batch)])
    rk = dr + np.einsum("gij,gj->gi", Ar, xs) + np.einsum("gij,gj->gi", Br, u)
    expect_d = rk - np.einsum("gij,gj->gi", Ag, xs) - np.einsum("gij,gj->gi", Bg, u)
    assert rel_err(d.cpu().numpy(), expect_d) <= 1e-12
    s.close()


# ------------------------------------------------------------------ one ADMM call (Sec. III-B)
def admm_case(prob, prec, iters_cold, iters_warm):
    x, u = perturbed_nominal(prob, seed=3, scale=0.02)
    Ar, Br, dr = oracle_linearize(prob, x, u)
    radius = np.full(prob.batch, 0.7)
    s = ucn.Solver(prob, precision=prec)
    xh, uh, res, st = s.admm_solve(t(x), t(u), t(Ar), t(Br), t(dr), t(radius), iters_cold, warm=False)
    xh2, uh2, res2, st2 = s.admm_solve(t(x), t(u), t(Ar), t(Br), t(dr), t(radius), iters_warm, warm=True)
    state = s.state_export().cpu().numpy()
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all() and (st2.cpu().numpy() == 0).all()
    mb = oracle.maxblk(prob)
    off = 0
    for b in range(prob.batch):
        N = int(prob.N[b])
        xo, uo = prob.xoff[b], prob.uoff[b]
        sl = lambda a, o, n: a[o:o + n]
        A_b, B_b, d_b = sl(Ar, uo, N), sl(Br, uo, N), sl(dr, uo, N)
        ref, r1, _ = oracle.problem_admm(prob, b, sl(x, xo, N + 1), sl(u, uo, N), A_b, B_b, d_b, radius[b], iters_cold)
        size = oracle.state_size(N, prob.nx, prob.nu, mb)
        yield b, "cold-xhat", xh.cpu().numpy()[xo:xo + N + 1], oracle.unpack_state(ref, N, prob.nx, prob.nu, mb)["xh"]
        yield b, "cold-res", res.cpu().numpy()[b], np.array(r1)
        ref2, r2, _ = oracle.problem_admm(prob, b, sl(x, xo, N + 1), sl(u, uo, N), A_b, B_b, d_b, radius[b], iters_warm, state=ref)
        yield b, "warm-state", state[off:off + size], ref2
        yield b, "warm-uhat", uh2.cpu().numpy()[uo:uo + N], oracle.unpack_state(ref2, N, prob.nx, prob.nu, mb)["uh"]
        yield b, "warm-res", res2.cpu().numpy()[b], np.array(r2)
        off += size
    s.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_admm_fp64_matches_oracle(name):
    for b, what, got, ref in admm_case(PROBLEMS[name](), ucn.UCN_PREC_FP64, 150, 60):
        assert rel_err(got, ref) <= TOL64, (b, what, rel_err(got, ref))


def residual_bound(prob, b, e):
    """Bound on |r_gpu - r_oracle| for the primal and dual residual norms of one
    instance, given e = the largest deviation of any ADMM iterate between the two
    paths.  |r_gpu - r_oracle| <= |v_gpu - v_oracle|_2 for the residual vectors v,
    whose m components are differences of iterates: primal ones (x - x-hat, x - z,
    z - (A x + B u + c), G xi - s) within (2 + |[A B]|_inf) e, dual ones
    (rho (new - old) of x-hat, z and the mirrors, and A^T of the neighbour's
    rho dz) within 2 rho (2 + |A|_1 + n_mirror) e."""
    N, nx, nu = int(prob.N[b]), prob.nx, prob.nu
    mb = oracle.maxblk(prob)
    x, u = perturbed_nominal(prob, seed=3, scale=0.02)
    A, B, _ = oracle_linearize(prob, x, u)
    uo = prob.uoff[b]
    Ab, Bb = A[uo:uo + N], B[uo:uo + N]
    ninf = max(np.abs(np.concatenate([Ab, Bb], axis=2)).sum(axis=2).max(), 0.0)
    n1 = np.abs(Ab).sum(axis=1).max()
    rho = max(prob.settings["rho_eq"], prob.settings["rho_dyn"], prob.settings["rho_geo"])
    m = (N + 1) * (nx + nu + 3 * mb)
    return (np.sqrt(m) * (2.0 + ninf) * e, np.sqrt(m) * 2.0 * rho * (2.0 + n1 + mb) * e)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_admm_fp32_matches_oracle(name):
    prob = PROBLEMS[name]()
    rows = list(admm_case(prob, ucn.UCN_PREC_FP32_REFINE, 150, 60))
    for b, what, got, ref in rows:
        if not what.endswith("res"):
            assert rel_err(got, ref) <= TOL32, (b, what, rel_err(got, ref))
    # the residual norms (summed in double-float from the FP32 iterates) differ from the
    # oracle's only through the iterates themselves
    for b in range(prob.batch):
        e = max(np.abs(np.asarray(g) - np.asarray(r)).max() for bb, w, g, r in rows if bb == b and w == "warm-state")
        bp, bd = residual_bound(prob, b, e)
        for bb, what, got, ref in rows:
            if bb == b and what.endswith("res"):
                assert abs(got[0] - ref[0]) <= bp, (b, what, got, ref, bp)
                assert abs(got[1] - ref[1]) <= bd, (b, what, got, ref, bd)


# ------------------------------------------------------------------ full SCP solve
def check_fp64_defects(prob, st, xg, ug):
    """The kernel's reported defect is an FP64 RK4 defect of exactly the doubles it
    returned: the oracle's RK4 on those doubles gives it to FP64 rounding."""
    d64 = oracle.traj_defects(prob, xg, ug)
    scale = np.array([max(1.0, np.abs(xg[prob.xoff[b]:prob.xoff[b] + prob.N[b] + 1]).max()) for b in range(prob.batch)])
    assert (np.abs(st["defect"] - d64) <= 1e-13 * scale).all(), np.abs(st["defect"] - d64).max()
    return d64


def scp_compare(prob, prec, tol, check_defect=False):
    """Every instance against the oracle's solve of the same inputs.  FP64: the
    same iterates (trajectories at 1e-9, identical accept flags and counts).
    FP32: trajectories at 1e-4 after the same number of SCP iterations (where the
    stop test landed on the other side of defect_tol the oracle is re-run to the
    GPU's count), and with check_defect every instance the oracle brings to the
    defect gate also passes it by the FP64 defect of the returned doubles."""
    s = ucn.Solver(prob, precision=prec)
    x, u = s.scp_solve()
    torch.cuda.synchronize()
    st = s.stats_host()
    xg, ug = x.cpu().numpy(), u.cpu().numpy()
    s.close()
    xr, ur, sr, _ = oracle.scp_solve(prob)
    d64 = check_fp64_defects(prob, st, xg, ug)
    if prec == ucn.UCN_PREC_FP64:
        for b in range(prob.batch):
            xo, uo, N = prob.xoff[b], prob.uoff[b], int(prob.N[b])
            assert rel_err(xg[xo:xo + N + 1], xr[xo:xo + N + 1]) <= tol, (b, rel_err(xg[xo:xo + N + 1], xr[xo:xo + N + 1]))
            assert rel_err(ug[uo:uo + N], ur[uo:uo + N]) <= tol, b
            assert int(st["scp_iters"][b]) == int(sr[b, 7])
            assert int(st["accepted"][b]) == int(sr[b, 8])
            assert int(st["accept_mask"][b]) == int(sr[b, 9])
            assert int(st["status"][b]) == int(sr[b, 10])
            assert abs(st["defect"][b] - sr[b, 0]) <= 1e-9 * max(1e-3, sr[b, 0])
            assert abs(st["cost"][b] - sr[b, 1]) <= 1e-9 * max(1.0, abs(sr[b, 1]))
    else:
        r = oracle.compare_batch(prob, xg, ug, st["scp_iters"], (xr, ur, sr), tol)
        assert r["summary"]["n_over_tol"] == 0, (r["summary"], r["err"])
    if check_defect:
        conv = sr[:, 0] <= 1e-5
        assert (d64[conv] <= 1e-5).all(), d64[conv].max()
        assert (st["status"][conv] == 0).all()
    return st, sr


def test_scp_fp64_quad_path_matches_oracle():
    # the single-quadrotor workload as stated: 15 SCP x 200 ADMM iterations, rho = 1
    scp_compare(W.quad_path(1, seed=0), ucn.UCN_PREC_FP64, TOL64)


def test_scp_fp64_quad_converging_matches_oracle():
    prob = W.quad_path(2, seed=0, settings=dict(rho_eq=10.0, rho_dyn=10.0, rho_geo=10.0, scp_iters=40, stop=1, step_tol=1.0))
    st, sr = scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)
    assert (sr[:, 0] <= 1e-5).all()


def test_scp_fp64_uneven_quad_matches_oracle():
    prob = W.quad_box(4, seed=7, N_range=(6, 30), obs_range=(3, 10), settings=dict(scp_iters=8, admm_iters=60))
    scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)


def test_scp_fp64_mars_matches_oracle():
    prob = W.mars_batch(3, seed=1, N=50, settings=dict(scp_iters=40, admm_iters=100))
    scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)


def test_scp_fp64_global_workspace_path_matches_oracle():
    # N = 60 quadrotor in FP64 does not fit in shared memory: per-node data in global memory
    prob = W.quad_path(1, seed=4, N=60, settings=dict(scp_iters=5, admm_iters=80))
    scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)


def test_scp_fp32_mars_fixed_iterations_matches_oracle():
    prob = W.mars_batch(4, seed=1, N=50, settings=dict(scp_iters=30, admm_iters=100, stop=0))
    scp_compare(prob, ucn.UCN_PREC_FP32_REFINE, TOL32)


def test_scp_fp32_mars_reaches_defect_gate():
    prob = W.mars_batch(6, seed=1)
    st, sr = scp_compare(prob, ucn.UCN_PREC_FP32_REFINE, TOL32, check_defect=True)
    assert (st["defect"] <= 1e-5).all()


def test_scp_fp64_quaternion_study_matches_oracle():
    # the 13-state study task (N = 50, 3 spheres, rho 1 -> 1e3 over 20 SCP x 100 ADMM iterations);
    # FP64 records of 17-row nodes exceed shared memory: global-memory workspace
    scp_compare(W.quat_study(2, seed=5), ucn.UCN_PREC_FP64, TOL64)


def test_scp_fp32_quaternion_study_matches_oracle():
    scp_compare(W.quat_study(3, seed=6), ucn.UCN_PREC_FP32_REFINE, TOL32)


def test_scp_fp32_quaternion_converges_to_the_defect_gate():
    prob = W.quat_study(3, rho0=10.0, rho_final=1e3, scp_iters=80, admm_iters=250, settings=dict(stop=1, step_tol=1.0))
    st, sr = scp_compare(prob, ucn.UCN_PREC_FP32_REFINE, TOL32, check_defect=True)
    assert (sr[:, 0] <= 1e-5).all()


def test_scp_fp64_mars6_matches_oracle():
    # the 6-DOF landing (glide slope, gimbal, tilt and body-rate sets), fixed 40 SCP iterations
    prob = W.mars6_batch(3, seed=7, settings=dict(scp_iters=40, stop=0))
    scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)


def test_scp_fp32_mars6_reaches_the_defect_gate():
    prob = W.mars6_batch(6, seed=7)
    st, sr = scp_compare(prob, ucn.UCN_PREC_FP32_REFINE, TOL32, check_defect=True)
    assert (sr[:, 0] <= 1e-5).all() and (st["defect"] <= 1e-5).all()


def test_scp_fp32_quad_matches_oracle():
    prob = W.quad_path(2, seed=0, settings=dict(rho_eq=10.0, rho_dyn=10.0, rho_geo=10.0, scp_iters=25))
    scp_compare(prob, ucn.UCN_PREC_FP32_REFINE, TOL32)


# ------------------------------------------------------------------ edge cases
def test_horizon_one_and_single_instance():
    prob = W.quad_path(1, seed=2, N=1, settings=dict(scp_iters=3, admm_iters=20))
    scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)


def test_longest_horizon():
    # 255 nodes: the largest CTA (256 threads)
    prob = W.mars_batch(1, seed=3, N=255, settings=dict(scp_iters=2, admm_iters=30, stop=0))
    scp_compare(prob, ucn.UCN_PREC_FP64, TOL64)


def test_full_size_mars_batch_sampled_against_oracle():
    # the Mars batch of 1024 instances in the benchmark's launch: every instance passes
    # the defect gate by the FP64 defect of its returned doubles (the kernel's own and the
    # oracle's RK4), and 64 evenly spaced instances match the oracle at 1e-4
    prob = W.mars_batch(1024, seed=1)
    s = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE)
    x, u = s.scp_solve()
    torch.cuda.synchronize()
    st = s.stats_host()
    xg, ug = x.cpu().numpy(), u.cpu().numpy()
    s.close()
    assert np.isfinite(xg).all() and np.isfinite(ug).all()
    assert (st["status"] == 0).all() and (st["defect"] <= 1e-5).all()
    d64 = check_fp64_defects(prob, st, xg, ug)
    assert (d64 <= 1e-5).all()
    idx = np.arange(64) * 16 + 7
    sub = prob.subset(idx)
    xs = np.concatenate([xg[prob.xoff[b]:prob.xoff[b] + 101] for b in idx])
    us = np.concatenate([ug[prob.uoff[b]:prob.uoff[b] + 100] for b in idx])
    ref = oracle.scp_solve(sub)[:3]
    r = oracle.compare_batch(sub, xs, us, st["scp_iters"][idx], ref, TOL32)
    assert r["summary"]["n_over_tol"] == 0, (r["summary"], r["err"])
    for b in idx:
        # every returned trajectory satisfies the boundary conditions exactly
        np.testing.assert_array_equal(xg[prob.xoff[b]], prob.xinit[b])
        np.testing.assert_array_equal(xg[prob.xoff[b] + 100][:6], 0.0)


def test_three_per_sm_first_round_gives_the_bits_of_a_solo_solve():
    # a 1024-instance Mars launch runs its first round (456 CTAs on 152 SMs) in the
    # three-CTAs-per-SM variant and the rest in the two-per-SM kernel; an instance
    # from each part gives the same bits as when it is solved alone (one CTA, the
    # two-per-SM kernel)
    prob = W.mars_batch(1024, seed=1, settings=dict(scp_iters=8, stop=0))
    s = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE)
    x, u = s.scp_solve()
    torch.cuda.synchronize()
    xg, ug, st = x.cpu().numpy(), u.cpu().numpy(), s.stats_host()
    assert ucn.ucn_problem_last_launches(s.handle) == 2
    s.close()
    for b in (0, 455, 456, 1023):
        one = prob.subset(np.array([b]))
        s1 = ucn.Solver(one, precision=ucn.UCN_PREC_FP32_REFINE)
        x1, u1 = s1.scp_solve()
        torch.cuda.synchronize()
        x1, u1, st1 = x1.cpu().numpy(), u1.cpu().numpy(), s1.stats_host()
        assert ucn.ucn_problem_last_launches(s1.handle) == 1
        s1.close()
        np.testing.assert_array_equal(x1, xg[prob.xoff[b]:prob.xoff[b] + 101])
        np.testing.assert_array_equal(u1, ug[prob.uoff[b]:prob.uoff[b] + 100])
        assert st1["accept_mask"][0] == st["accept_mask"][b] and st1["defect"][0] == st["defect"][b]


# ------------------------------------------------------------------ two threads per node (3-DOF Mars, FP32)
def solve_with_lanes(prob, lanes, prec=ucn.UCN_PREC_FP32_REFINE):
    s = ucn.Solver(prob, precision=prec)
    ucn.ucn_problem_set_lanes(s.handle, lanes)
    assert ucn.ucn_problem_lanes(s.handle) == lanes
    x, u = s.scp_solve()
    torch.cuda.synchronize()
    st = s.stats_host()
    out = x.cpu().numpy(), u.cpu().numpy(), st
    s.close()
    return out


@pytest.mark.parametrize("case", ["batch", "uneven", "shortest", "longest"])
def test_pair_kernel_matches_oracle(case):
    # the pair kernel (2 threads per node) against the oracle at 1e-4 after the same
    # SCP iteration count, and against the one-thread kernel
    if case == "batch":
        prob = W.mars_batch(48, seed=1)
    elif case == "uneven":
        # horizons 5..111 in one launch: inactive pairs and partly filled warps
        base = W.mars_batch(1, seed=2, N=111)
        probs = [W.mars_batch(1, seed=20 + k, N=n) for k, n in enumerate((5, 37, 64, 111, 90, 17))]
        prob = probs[0]
        for p in probs[1:]:
            prob = concat(prob, p)
    elif case == "shortest":
        prob = W.mars_batch(3, seed=4, N=1, settings=dict(scp_iters=4, admm_iters=30, stop=0))
    else:
        prob = W.mars_batch(4, seed=5, N=111)
    xg, ug, st = solve_with_lanes(prob, 2)
    ref = oracle.scp_solve(prob)[:3]
    r = oracle.compare_batch(prob, xg, ug, st["scp_iters"], ref, TOL32)
    assert r["summary"]["n_over_tol"] == 0, (r["summary"], r["err"])
    d64 = check_fp64_defects(prob, st, xg, ug)
    conv = ref[2][:, 0] <= 1e-5
    assert (d64[conv] <= 1e-5).all() and (st["status"][conv] == 0).all()
    x1, u1, st1 = solve_with_lanes(prob, 1)
    same = st1["scp_iters"] == st["scp_iters"]
    for b in np.nonzero(same)[0]:
        xo, N = prob.xoff[b], int(prob.N[b])
        assert rel_err(xg[xo:xo + N + 1], x1[xo:xo + N + 1]) <= TOL32


def concat(a, b):
    import dataclasses
    f = {}
    for fld in dataclasses.fields(a):
        va, vb = getattr(a, fld.name), getattr(b, fld.name)
        if fld.name in ("model", "nx", "nu"):
            f[fld.name] = va
        elif fld.name == "settings":
            f[fld.name] = dict(va)
        else:
            f[fld.name] = np.concatenate([va, vb])
    return W.Problem(**f)


def test_pair_layout_is_refused_where_it_does_not_apply():
    with pytest.raises(ucn.UcnError):
        solve_with_lanes(W.mars_batch(1, seed=1, N=20), 2, prec=ucn.UCN_PREC_FP64)
    with pytest.raises(ucn.UcnError):
        solve_with_lanes(W.mars_batch(1, seed=1, N=112), 2)      # 113 nodes: beyond the pair kernel's CTA
    with pytest.raises(ucn.UcnError):
        solve_with_lanes(W.quad_path(1, seed=0, N=20), 2)


# ------------------------------------------------------------------ warm start from a kept ADMM state
def shifted(prob, dr):
    """The same instances with the initial position moved by dr (non-dimensional)."""
    q = prob.subset(np.arange(prob.batch))
    q.xinit = q.xinit.copy()
    q.xinit[:, 0:3] += dr
    return q


@pytest.mark.parametrize("prec,tol", [(ucn.UCN_PREC_FP64, TOL64), (ucn.UCN_PREC_FP32_REFINE, TOL32)])
def test_warm_start_from_kept_state_matches_oracle(prec, tol):
    # solve, keep the final ADMM state and trajectory, then solve from that state (at
    # the schedule's final penalties): (1) the problem with its initial position moved
    # (the next request of a stream, or the next MPC step) against the oracle started
    # from the same state and guess; (2) the same problem again, which stops at once,
    # in fewer SCP iterations than a start from the kept trajectory alone
    prob = W.mars_batch(4, seed=11, N=60)
    s = ucn.Solver(prob, precision=prec)
    x1, u1 = s.scp_solve()
    state = s.state_export()
    torch.cuda.synchronize()
    x1h, u1h = x1.cpu().numpy().copy(), u1.cpu().numpy().copy()
    s.close()
    p2 = shifted(prob, np.array([0.005, -0.003, 0.002]))
    s2 = ucn.Solver(p2, precision=prec)
    xg, ug = s2.tensor(x1h), s2.tensor(u1h)
    xw, uw = s2.scp_solve(xg, ug, state=state)
    torch.cuda.synchronize()
    xw, uw, stw = xw.cpu().numpy(), uw.cpu().numpy(), s2.stats_host()
    s2.close()
    xr, ur, sr = oracle.scp_solve_warm(p2, state.cpu().numpy(), xguess=x1h, uguess=u1h)
    np.testing.assert_array_equal(stw["scp_iters"], sr[:, 7].astype(int))
    for b in range(p2.batch):
        xo, uo, N = p2.xoff[b], p2.uoff[b], int(p2.N[b])
        assert rel_err(xw[xo:xo + N + 1], xr[xo:xo + N + 1]) <= tol, (b, rel_err(xw[xo:xo + N + 1], xr[xo:xo + N + 1]))
        assert rel_err(uw[uo:uo + N], ur[uo:uo + N]) <= tol, b
    s3 = ucn.Solver(prob, precision=prec)
    xg, ug = s3.tensor(x1h), s3.tensor(u1h)
    s3.scp_solve(xg, ug, state=state)
    torch.cuda.synchronize()
    st_state = s3.stats_host()
    s3.scp_solve(xg, ug)                  # the kept trajectory alone (cold ADMM state)
    torch.cuda.synchronize()
    st_traj = s3.stats_host()
    s3.close()
    assert (st_state["defect"] <= 1e-5).all() and (st_state["status"] == 0).all()
    assert st_state["scp_iters"].mean() < st_traj["scp_iters"].mean(), (st_state["scp_iters"], st_traj["scp_iters"])
