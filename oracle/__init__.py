"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct implementation of the method of
arXiv 2603.10711 (SCP with a consensus-ADMM inner solver), in C++
(``ucn_oracle.cpp``), FP64, plain loops.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this package.  The CUDA library never loads it, and the two share
no code: each side has its own headers, structures and helpers; only the
seeded generators in ``workloads`` feed both.

Every function cites the passage of the paper it follows; the pins in
``tests/test_oracle_*.py`` tie it to mathematics other than itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucn_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

NSTAT = 16
NLOG = 8
BLK_NONE, BLK_HALF, BLK_BALL, BLK_CONE = -1, 0, 1, 2
STAT_NAMES = ["defect", "cost", "merit", "primal", "dual", "radius", "step",
              "iters", "accepted", "accept_mask", "status"]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain C++17, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               _SRC, "-o", _LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_longlong)
_up = C.POINTER(C.c_ubyte)


class OrcProblem(C.Structure):
    _fields_ = [
        ("model", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("batch", C.c_int),
        ("N", _ip), ("xoff", _lp), ("uoff", _lp), ("dt", _dp), ("params", _dp),
        ("Qd", _dp), ("xref", _dp), ("Rd", _dp), ("uref", _dp), ("QNd", _dp), ("qN", _dp),
        ("xlo", _dp), ("xhi", _dp), ("ulo", _dp), ("uhi", _dp),
        ("xinit", _dp), ("xtarget", _dp), ("tmask", _up),
        ("max_obs", C.c_int), ("nobs", _ip), ("obs_c", _dp), ("obs_r", _dp), ("sets", _dp),
        ("rho_eq", C.c_double), ("rho_dyn", C.c_double), ("rho_geo", C.c_double), ("rho_final", C.c_double),
        ("scp_iters", C.c_int), ("admm_iters", C.c_int), ("stop", C.c_int),
        ("tr_init", C.c_double), ("tr_min", C.c_double), ("tr_max", C.c_double), ("w_d", C.c_double),
        ("defect_tol", C.c_double), ("step_tol", C.c_double), ("vc_weight", C.c_double),
        ("group", C.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_state_size.restype = C.c_int
            _lib.orc_admm_qp.restype = C.c_int
            _lib.orc_problem_admm.restype = C.c_int
            _lib.orc_max_threads.restype = C.c_int
            _lib.orc_rk4.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp, _dp]
            _lib.orc_f.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
            _lib.orc_linearize.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp, _dp, _dp, _dp, _dp]
            _lib.orc_jac_complex_step.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp, _dp, _dp]
            _lib.orc_project.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp]
            _lib.orc_scp_solve_iters.restype = C.c_int
            _lib.orc_traj_defects.restype = C.c_int
            _lib.orc_scp_solve_warm.restype = C.c_int
        return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def model_dims(model: int):
    return {1: (12, 4), 2: (7, 3), 3: (13, 4), 4: (14, 3)}[int(model)]


def f(model, params, x, u):
    """Continuous dynamics f(x, u)."""
    nx, _ = model_dims(model)
    out = np.zeros(nx)
    lib().orc_f(model, _d(_f64(params)), _d(_f64(x)), _d(_f64(u)), _d(out))
    return out


def rk4(model, params, h, x, u):
    """One RK4 step of length h (Eq. (1b))."""
    nx, _ = model_dims(model)
    out = np.zeros(nx)
    lib().orc_rk4(model, _d(_f64(params)), float(h), _d(_f64(x)), _d(_f64(u)), _d(out))
    return out


def linearize(model, params, h, x, u):
    """(A, B, d, x_next) of Eq. (2b) about (x, u) by the RK4 variational equations."""
    nx, nu = model_dims(model)
    A = np.zeros((nx, nx)); B = np.zeros((nx, nu)); d = np.zeros(nx); xn = np.zeros(nx)
    lib().orc_linearize(model, _d(_f64(params)), float(h), _d(_f64(x)), _d(_f64(u)), _d(A), _d(B), _d(d), _d(xn))
    return A, B, d, xn


def jac_complex_step(model, params, h, x, u):
    nx, nu = model_dims(model)
    A = np.zeros((nx, nx)); B = np.zeros((nx, nu))
    lib().orc_jac_complex_step(model, _d(_f64(params)), float(h), _d(_f64(x)), _d(_f64(u)), _d(A), _d(B))
    return A, B


def project(kind: int, p0: float, y):
    y = _f64(y)
    out = np.zeros_like(y)
    lib().orc_project(int(kind), int(y.size), float(p0), _d(y), _d(out))
    return out


def state_size(N, nx, nu, mb):
    return 6 * (N + 1) * nx + 3 * N * nu + 2 * (N + 1) * mb * 3


def unpack_state(flat, N, nx, nu, mb):
    """Split the flat ADMM state (order x, u, z, lam, mu, xh, uh, nux, nuu, s, nus)."""
    sizes = [("x", (N + 1, nx)), ("u", (N, nu)), ("z", (N + 1, nx)), ("lam", (N + 1, nx)),
             ("mu", (N + 1, nx)), ("xh", (N + 1, nx)), ("uh", (N, nu)), ("nux", (N + 1, nx)),
             ("nuu", (N, nu)), ("s", (N + 1, mb, 3)), ("nus", (N + 1, mb, 3))]
    out, o = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def admm_qp(qp: dict, iters: int, state=None, xbar=None, ubar=None, rho=(1.0, 1.0, 1.0)):
    """Generic QP ADMM (Steps 1-4 of Sec. III-B) on explicit per-node data.

    ``qp`` keys: N, nx, nu, A, B, d, Q, R, M, q, r, xlo, xhi, ulo, uhi, x0,
    tmask, xtarget, and optionally blk_kind [(N+1),mb], blk_G [(N+1),mb,3,nx+nu],
    blk_p [(N+1),mb].  Returns (state_flat, (primal, dual), status).
    """
    N, nx, nu = qp["N"], qp["nx"], qp["nu"]
    mb = qp.get("blk_kind", np.zeros((N + 1, 0))).shape[1]
    kind = np.ascontiguousarray(qp.get("blk_kind", np.zeros((N + 1, 0))), dtype=np.int32)
    G = _f64(qp.get("blk_G", np.zeros((N + 1, mb, 3, nx + nu))))
    p0 = _f64(qp.get("blk_p", np.zeros((N + 1, mb))))
    st = np.zeros(state_size(N, nx, nu, mb)) if state is None else _f64(state).copy()
    warm = 0 if state is None else 1
    if xbar is None:
        xbar = np.zeros((N + 1, nx))
    if ubar is None:
        ubar = np.zeros((N, nu))
    tm = np.ascontiguousarray(qp.get("tmask", np.zeros(nx)), dtype=np.uint8)
    xt = _f64(qp.get("xtarget", np.zeros(nx)))
    stats = np.zeros(2)
    arrs = [_f64(qp[k]) for k in ("A", "B", "d", "Q", "R", "M", "q", "r", "xlo", "xhi", "ulo", "uhi", "x0")]
    xb, ub = _f64(xbar), _f64(ubar)
    rc = lib().orc_admm_qp(
        C.c_int(N), C.c_int(nx), C.c_int(nu), *[_d(a) for a in arrs[:12]], _d(arrs[12]),
        tm.ctypes.data_as(_up), _d(xt), C.c_int(mb), kind.ctypes.data_as(_ip), _d(G), _d(p0),
        C.c_double(rho[0]), C.c_double(rho[1]), C.c_double(rho[2]), C.c_int(iters), C.c_int(warm),
        _d(xb), _d(ub), _d(st), _d(stats))
    return st, tuple(stats), rc


class _Pinned:
    """Keeps the numpy arrays behind an OrcProblem alive."""

    def __init__(self, prob):
        self.prob = prob
        p = prob
        self.arrs = {}

        def keep(name, a, dt=np.float64):
            a = np.ascontiguousarray(a, dtype=dt)
            self.arrs[name] = a
            return a

        s = p.settings
        o = OrcProblem()
        o.model, o.nx, o.nu, o.batch = p.model, p.nx, p.nu, p.batch
        o.N = keep("N", p.N, np.int32).ctypes.data_as(_ip)
        o.xoff = keep("xoff", p.xoff, np.int64).ctypes.data_as(_lp)
        o.uoff = keep("uoff", p.uoff, np.int64).ctypes.data_as(_lp)
        for name in ("dt", "params", "Qd", "xref", "Rd", "uref", "QNd", "qN", "xlo", "xhi", "ulo", "uhi",
                     "xinit", "xtarget", "obs_c", "obs_r", "sets"):
            setattr(o, name, _d(keep(name, getattr(p, name))))
        o.tmask = keep("tmask", p.tmask, np.uint8).ctypes.data_as(_up)
        o.max_obs = p.max_obs
        o.nobs = keep("nobs", p.nobs, np.int32).ctypes.data_as(_ip)
        o.rho_eq, o.rho_dyn, o.rho_geo = float(s["rho_eq"]), float(s["rho_dyn"]), float(s["rho_geo"])
        o.rho_final = float(s.get("rho_final", 0.0))
        o.scp_iters, o.admm_iters, o.stop = int(s["scp_iters"]), int(s["admm_iters"]), int(s.get("stop", 0))
        o.tr_init, o.tr_min, o.tr_max = float(s["tr_init"]), float(s["tr_min"]), float(s["tr_max"])
        o.w_d, o.defect_tol, o.step_tol = float(s["w_d"]), float(s["defect_tol"]), float(s["step_tol"])
        o.vc_weight = float(s.get("vc_weight", 0.0))
        o.group = int(s.get("group", 1))
        self.c = o


def maxblk(prob):
    return {2: 3, 4: 6}.get(int(prob.model), prob.max_obs)


def problem_admm(prob, b, xbar, ubar, A, B, d, radius, iters, state=None):
    """ADMM on instance b's SCP subproblem (Eq. (2)) at the given linearisation."""
    pin = _Pinned(prob)
    N, nx, nu = int(prob.N[b]), prob.nx, prob.nu
    st = np.zeros(state_size(N, nx, nu, maxblk(prob))) if state is None else _f64(state).copy()
    stats = np.zeros(2)
    rc = lib().orc_problem_admm(C.byref(pin.c), C.c_int(b), _d(_f64(xbar)), _d(_f64(ubar)), _d(_f64(A)),
                                _d(_f64(B)), _d(_f64(d)), C.c_double(radius), C.c_int(iters),
                                C.c_int(0 if state is None else 1), _d(st), _d(stats))
    return st, tuple(stats), rc


def scp_solve(prob, nthreads: int = 0, xguess=None, uguess=None, log=False):
    """Full SCP solve of every instance.  Returns (x, u, stats[B,16], log[B,K,8] or None)."""
    pin = _Pinned(prob)
    xg = _f64(prob.xguess if xguess is None else xguess)
    ug = _f64(prob.uguess if uguess is None else uguess)
    xo = np.zeros_like(xg); uo = np.zeros_like(ug)
    st = np.zeros((prob.batch, NSTAT))
    K = int(prob.settings["scp_iters"])
    lg = np.full((prob.batch, K, NLOG), np.nan) if log else None
    lib().orc_scp_solve(C.byref(pin.c), _d(xg), _d(ug), _d(xo), _d(uo), _d(st),
                        _d(lg) if log else _dp(), C.c_int(nthreads))
    return xo, uo, st, lg


def scp_solve_iters(prob, run_iters, nthreads: int = 0, xguess=None, uguess=None):
    """SCP solve with exactly ``run_iters[b]`` SCP iterations per instance
    (per scenario group: its first instance's entry), without the stop test and
    with the penalty schedule of the cap.  Returns (x, u, stats[B,16])."""
    pin = _Pinned(prob)
    xg = _f64(prob.xguess if xguess is None else xguess)
    ug = _f64(prob.uguess if uguess is None else uguess)
    xo = np.zeros_like(xg); uo = np.zeros_like(ug)
    st = np.zeros((prob.batch, NSTAT))
    ri = np.ascontiguousarray(run_iters, dtype=np.int32)
    assert ri.shape == (prob.batch,)
    lib().orc_scp_solve_iters(C.byref(pin.c), _d(xg), _d(ug), _d(xo), _d(uo), _d(st),
                              ri.ctypes.data_as(_ip), C.c_int(nthreads))
    return xo, uo, st


def scp_solve_warm(prob, state, nthreads: int = 0, xguess=None, uguess=None):
    """SCP solve of independent instances started from the ADMM ``state`` (the
    instances' flat absolute states, one after the other) instead of the cold
    start.  Returns (x, u, stats[B,16])."""
    pin = _Pinned(prob)
    xg = _f64(prob.xguess if xguess is None else xguess)
    ug = _f64(prob.uguess if uguess is None else uguess)
    xo = np.zeros_like(xg); uo = np.zeros_like(ug)
    st = np.zeros((prob.batch, NSTAT))
    if lib().orc_scp_solve_warm(C.byref(pin.c), _d(xg), _d(ug), _d(_f64(state)), _d(xo), _d(uo), _d(st),
                                C.c_int(nthreads)) != 0:
        raise ValueError("scenario groups start cold")
    return xo, uo, st


def traj_defects(prob, x, u):
    """max_i |RK4(x_i, u_i) - x_{i+1}|_inf per instance of packed trajectories, FP64."""
    pin = _Pinned(prob)
    out = np.zeros(prob.batch)
    lib().orc_traj_defects(C.byref(pin.c), _d(_f64(x)), _d(_f64(u)), _d(out))
    return out


def rel_err(a, b):
    """Normwise relative difference with floor 1: |a - b|_max / max(1, |b|_max)."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max())) if b.size else 0.0


def compare_batch(prob, x, u, iters, ref, tol, nthreads: int = 0):
    """Element-by-element parity of packed trajectories (x, u) that ran
    ``iters[b]`` SCP iterations against the oracle's solve ``ref = (xr, ur, sr)``
    of the same inputs.  The stop test (max defect <= defect_tol) is a decision
    on a floating-point value: where the two solves stopped after different
    iteration counts, both stopping points are valid and the unique object to
    compare is the trajectory after the same count, so the oracle is re-run to
    exactly ``iters[b]`` iterations for those instances.  Returns a dict with
    per-instance errors and a summary."""
    xr, ur, sr = ref[0], ref[1], ref[2]
    iters = np.asarray(iters).astype(np.int64)
    mism = np.nonzero(iters != sr[:, 7].astype(np.int64))[0]
    K = int(prob.settings.get("group", 1))
    if K > 1 and mism.size:       # whole scenario groups
        mism = np.unique(np.concatenate([np.arange(g * K, (g + 1) * K) for g in np.unique(mism // K)]))
    xr = xr.copy(); ur = ur.copy()
    if mism.size:
        sub = prob.subset(mism)
        xs, us, _ = scp_solve_iters(sub, iters[mism], nthreads=nthreads)
        for k, b in enumerate(mism):
            xr[prob.xoff[b]:prob.xoff[b] + prob.N[b] + 1] = xs[sub.xoff[k]:sub.xoff[k] + sub.N[k] + 1]
            ur[prob.uoff[b]:prob.uoff[b] + prob.N[b]] = us[sub.uoff[k]:sub.uoff[k] + sub.N[k]]
    err = np.zeros(prob.batch)
    for b in range(prob.batch):
        xo, uo, N = prob.xoff[b], prob.uoff[b], int(prob.N[b])
        err[b] = max(rel_err(x[xo:xo + N + 1], xr[xo:xo + N + 1]), rel_err(u[uo:uo + N], ur[uo:uo + N]))
    d64 = traj_defects(prob, x, u)
    return {"err": err, "mismatch": mism, "fp64_defect": d64,
            "summary": {"instances": int(prob.batch), "tol": tol, "max_rel_err": float(err.max()) if err.size else 0.0,
                        "n_over_tol": int(np.sum(err > tol)), "scp_iters_mismatch": int(mism.size),
                        "fp64_defect_max": float(d64.max()) if d64.size else 0.0,
                        "n_fp64_defect_over_tol": int(np.sum(d64 > prob.settings["defect_tol"]))}}


def max_threads() -> int:
    return int(lib().orc_max_threads())
