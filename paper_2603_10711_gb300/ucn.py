"""Thin Python binding of the ucn C ABI (include/ucn.h).

Argument marshalling only: every step of the method runs in the CUDA
library ``libucn.so`` built in-tree by ``build.py``.  There is no fallback:
if the library is missing or no GPU is present, the calls raise.

Device buffers are torch CUDA tensors (float64 / int32, contiguous); the
stream is torch's current stream unless one is given.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libucn.so")

UCN_OK, UCN_EINVAL, UCN_ENOMEM, UCN_ECUDA, UCN_ENUMERIC, UCN_ENOTCONV, UCN_ETIMEOUT, UCN_EBUSY = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENUMERIC", 5: "ENOTCONV", 6: "ETIMEOUT", 7: "EBUSY"}
UCN_MODEL_QUAD12, UCN_MODEL_MARS7, UCN_MODEL_QUAT13, UCN_MODEL_MARS14 = 1, 2, 3, 4
UCN_PREC_FP64, UCN_PREC_FP32_REFINE = 0, 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_up = C.POINTER(C.c_ubyte)


class ProblemDesc(C.Structure):
    """Mirror of ucn_problem_desc."""
    _fields_ = [
        ("model", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("batch", C.c_int),
        ("horizon", _ip), ("dt", _dp), ("model_params", _dp),
        ("Q_diag", _dp), ("x_ref", _dp), ("R_diag", _dp), ("u_ref", _dp), ("QN_diag", _dp), ("qN", _dp),
        ("x_lo", _dp), ("x_hi", _dp), ("u_lo", _dp), ("u_hi", _dp),
        ("x_init", _dp), ("x_target", _dp), ("term_mask", _up),
        ("max_obs", C.c_int), ("n_obs", _ip), ("obs_c", _dp), ("obs_r", _dp), ("sets", _dp),
        ("rho_eq", C.c_double), ("rho_dyn", C.c_double), ("rho_geo", C.c_double), ("rho_final", C.c_double),
        ("scp_iters", C.c_int), ("admm_iters", C.c_int), ("stop", C.c_int),
        ("tr_init", C.c_double), ("tr_min", C.c_double), ("tr_max", C.c_double), ("w_d", C.c_double),
        ("defect_tol", C.c_double), ("step_tol", C.c_double), ("vc_weight", C.c_double),
        ("precision", C.c_int), ("timeout_s", C.c_double), ("group", C.c_int),
    ]


# Mirror of ucn_scp_stats (128 bytes).
STATS_DTYPE = np.dtype([
    ("defect", "f8"), ("cost", "f8"), ("merit", "f8"), ("primal_res", "f8"), ("dual_res", "f8"),
    ("tr_radius", "f8"), ("step", "f8"), ("scp_iters", "i4"), ("accepted", "i4"), ("accept_mask", "u8"),
    ("status", "i4"), ("reserved", "i4"), ("t_start_ns", "u8"), ("t_end_ns", "u8"), ("pad", "f8", (4,)),
])
assert STATS_DTYPE.itemsize == 128

_lib = None
_lock = threading.Lock()


class UcnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def lib():
    """Load libucn.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libucn.so is missing; build it with paper_2603_10711_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp = C.c_void_p
            L.ucn_last_error.restype = C.c_char_p
            L.ucn_problem_create.argtypes = [C.POINTER(ProblemDesc), C.POINTER(vp)]
            L.ucn_problem_create.restype = C.c_int
            L.ucn_problem_destroy.argtypes = [vp]
            L.ucn_problem_destroy.restype = None
            for f in ("ucn_total_x", "ucn_total_u", "ucn_state_size"):
                getattr(L, f).argtypes = [vp]
                getattr(L, f).restype = C.c_longlong
            L.ucn_problem_set_order.argtypes = [vp, _ip]
            L.ucn_problem_set_order.restype = C.c_int
            L.ucn_problem_set_lanes.argtypes = [vp, C.c_int]
            L.ucn_problem_set_lanes.restype = C.c_int
            L.ucn_problem_lanes.argtypes = [vp]
            L.ucn_problem_lanes.restype = C.c_int
            L.ucn_problem_last_launches.argtypes = [vp]
            L.ucn_problem_last_launches.restype = C.c_int
            L.ucn_linearize.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            L.ucn_linearize.restype = C.c_int
            L.ucn_admm_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp, vp, vp]
            L.ucn_admm_solve.restype = C.c_int
            L.ucn_state_export.argtypes = [vp, vp, vp]
            L.ucn_state_export.restype = C.c_int
            L.ucn_scp_solve.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.ucn_scp_solve.restype = C.c_int
            L.ucn_scp_solve_warm.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.ucn_scp_solve_warm.restype = C.c_int
            L.ucn_mpc_shift.argtypes = [vp, vp, vp, vp, vp, vp]
            L.ucn_mpc_shift.restype = C.c_int
            L.ucn_scp_solve_noalloc.argtypes = [C.POINTER(ProblemDesc), vp, vp, vp, vp, vp, vp, vp]
            L.ucn_scp_solve_noalloc.restype = C.c_int
            L.ucn_df_check.argtypes = [C.c_int, vp, vp, vp, C.c_double, C.c_longlong, vp, vp]
            L.ucn_df_check.restype = C.c_int
            _lib = L
        return _lib


def ucn_last_error() -> str:
    return lib().ucn_last_error().decode()


def _check(rc):
    if rc != UCN_OK:
        raise UcnError(rc, ucn_last_error())


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t, dtype=None, numel=None, name="buffer"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s holds %d elements, needs %d" % (name, t.numel(), numel))
    return C.c_void_p(t.data_ptr())


class _Keep:
    """Host arrays referenced by a ProblemDesc while ucn_problem_create copies them."""

    def __init__(self):
        self.arrays = []

    def d(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.arrays.append(a)
        return a.ctypes.data_as(_dp)

    def i(self, a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        self.arrays.append(a)
        return a.ctypes.data_as(_ip)

    def u8(self, a):
        a = np.ascontiguousarray(a, dtype=np.uint8)
        self.arrays.append(a)
        return a.ctypes.data_as(_up)


def make_desc(prob, precision=UCN_PREC_FP64, timeout_s=0.0, **overrides):
    """ucn_problem_desc from any object with the workload-generator fields
    (model, nx, nu, N, dt, params, Qd, ... , settings)."""
    k = _Keep()
    s = dict(prob.settings)
    s.update(overrides)
    d = ProblemDesc()
    d.model, d.nx, d.nu, d.batch = int(prob.model), int(prob.nx), int(prob.nu), int(len(prob.N))
    d.horizon = k.i(prob.N)
    d.dt = k.d(prob.dt)
    d.model_params = k.d(prob.params)
    d.Q_diag, d.x_ref, d.R_diag, d.u_ref = k.d(prob.Qd), k.d(prob.xref), k.d(prob.Rd), k.d(prob.uref)
    d.QN_diag, d.qN = k.d(prob.QNd), k.d(prob.qN)
    d.x_lo, d.x_hi, d.u_lo, d.u_hi = k.d(prob.xlo), k.d(prob.xhi), k.d(prob.ulo), k.d(prob.uhi)
    d.x_init, d.x_target, d.term_mask = k.d(prob.xinit), k.d(prob.xtarget), k.u8(prob.tmask)
    d.max_obs = int(prob.obs_r.shape[1])
    d.n_obs = k.i(prob.nobs)
    d.obs_c = k.d(prob.obs_c if prob.obs_c.size else np.zeros(1))
    d.obs_r = k.d(prob.obs_r if prob.obs_r.size else np.zeros(1))
    d.sets = k.d(prob.sets)
    d.rho_eq, d.rho_dyn, d.rho_geo = float(s["rho_eq"]), float(s["rho_dyn"]), float(s["rho_geo"])
    d.rho_final = float(s.get("rho_final", 0.0))
    d.scp_iters, d.admm_iters, d.stop = int(s["scp_iters"]), int(s["admm_iters"]), int(s.get("stop", 0))
    d.tr_init, d.tr_min, d.tr_max = float(s["tr_init"]), float(s["tr_min"]), float(s["tr_max"])
    d.w_d, d.defect_tol, d.step_tol = float(s["w_d"]), float(s["defect_tol"]), float(s["step_tol"])
    d.vc_weight = float(s.get("vc_weight", 0.0))
    d.precision = int(precision)
    d.timeout_s = float(timeout_s)
    d.group = int(s.get("group", 1))
    return d, k


def ucn_problem_create(desc: ProblemDesc):
    h = C.c_void_p()
    _check(lib().ucn_problem_create(C.byref(desc), C.byref(h)))
    return h


def ucn_problem_destroy(h):
    lib().ucn_problem_destroy(h)


def ucn_problem_set_lanes(h, lanes_per_node):
    """Threads per node of the fused solve (1, or 4 for quadrotor problems)."""
    _check(lib().ucn_problem_set_lanes(h, int(lanes_per_node)))


def ucn_problem_lanes(h):
    return int(lib().ucn_problem_lanes(h))


def ucn_problem_last_launches(h):
    return int(lib().ucn_problem_last_launches(h))


def ucn_problem_set_order(h, order=None):
    """CTA -> instance order of the fused solve (None: instance order)."""
    if order is None:
        _check(lib().ucn_problem_set_order(h, None))
    else:
        o = np.ascontiguousarray(order, dtype=np.int32)
        _check(lib().ucn_problem_set_order(h, o.ctypes.data_as(_ip)))


def ucn_total_x(h):
    return int(lib().ucn_total_x(h))


def ucn_total_u(h):
    return int(lib().ucn_total_u(h))


def ucn_state_size(h):
    return int(lib().ucn_state_size(h))


def ucn_linearize(h, xbar, ubar, A, B, d, stream=None):
    import torch
    f = torch.float64
    _check(lib().ucn_linearize(h, _ptr(xbar, f, name="xbar"), _ptr(ubar, f, name="ubar"), _ptr(A, f, name="A"),
                               _ptr(B, f, name="B"), _ptr(d, f, name="d"), _stream(stream)))


def ucn_admm_solve(h, xbar, ubar, A, B, d, radius, iters, warm, xhat, uhat, res, status, stream=None):
    import torch
    f = torch.float64
    _check(lib().ucn_admm_solve(h, _ptr(xbar, f), _ptr(ubar, f), _ptr(A, f), _ptr(B, f), _ptr(d, f), _ptr(radius, f),
                                int(iters), int(warm), _ptr(xhat, f), _ptr(uhat, f), _ptr(res, f),
                                _ptr(status, torch.int32), _stream(stream)))


def ucn_state_export(h, out, stream=None):
    import torch
    _check(lib().ucn_state_export(h, _ptr(out, torch.float64, ucn_state_size(h), "state"), _stream(stream)))


def ucn_scp_solve(h, x0, u0, x_out, u_out, stats, status, stream=None):
    import torch
    f = torch.float64
    _check(lib().ucn_scp_solve(h, _ptr(x0, f, name="x0"), _ptr(u0, f, name="u0"), _ptr(x_out, f, name="x_out"),
                               _ptr(u_out, f, name="u_out"), _ptr(stats, torch.uint8, name="stats"),
                               _ptr(status, torch.int32, name="status"), _stream(stream)))


def ucn_scp_solve_warm(h, x0, u0, state, x_out, u_out, stats, status, stream=None):
    """ucn_scp_solve started from an exported ADMM state (``state``: float64,
    ucn_state_size elements)."""
    import torch
    f = torch.float64
    _check(lib().ucn_scp_solve_warm(h, _ptr(x0, f, name="x0"), _ptr(u0, f, name="u0"),
                                    _ptr(state, f, ucn_state_size(h), "state"), _ptr(x_out, f, name="x_out"),
                                    _ptr(u_out, f, name="u_out"), _ptr(stats, torch.uint8, name="stats"),
                                    _ptr(status, torch.int32, name="status"), _stream(stream)))


def ucn_mpc_shift(h, x, u, xg, ug, stream=None):
    """Apply the (shared) first control to the plant and shift the solution
    into the next warm start; updates the problem's initial states."""
    import torch
    f = torch.float64
    _check(lib().ucn_mpc_shift(h, _ptr(x, f, name="x"), _ptr(u, f, name="u"), _ptr(xg, f, name="xg"),
                               _ptr(ug, f, name="ug"), _stream(stream)))


UCN_DF_ADD, UCN_DF_SUB, UCN_DF_MUL, UCN_DF_DIV, UCN_DF_SQRT, UCN_DF_ROUND, UCN_DF_RK4 = 0, 1, 2, 3, 4, 5, 100
UCN_DF_SQDIFF_SUM, UCN_DF_SQ_SUM = 6, 7


def ucn_df_check(op, a, b, prm, h, out, stream=None):
    """The FP32 path's double-float arithmetic on device FP64 tensors (see
    include/ucn.h): elementwise ops on a, b, or one RK4 step per row."""
    import torch
    f = torch.float64
    n = a.numel() if op in (UCN_DF_SQDIFF_SUM, UCN_DF_SQ_SUM) else out.numel() if op < UCN_DF_RK4 else out.shape[0]
    _check(lib().ucn_df_check(int(op), _ptr(a, f, name="a"), None if b is None else _ptr(b, f, name="b"),
                              None if prm is None else _ptr(prm, f, name="prm"), float(h), int(n),
                              _ptr(out, f, name="out"), _stream(stream)))


def ucn_scp_solve_noalloc(desc: ProblemDesc, x0, u0, x_out, u_out, stats, status, stream=None):
    """No-allocation solve: ``desc`` holds a host ``horizon`` array and device
    pointers for every other array (see include/ucn.h)."""
    import torch
    f = torch.float64
    _check(lib().ucn_scp_solve_noalloc(C.byref(desc), _ptr(x0, f, name="x0"), _ptr(u0, f, name="u0"),
                                       _ptr(x_out, f, name="x_out"), _ptr(u_out, f, name="u_out"),
                                       _ptr(stats, torch.uint8, name="stats"), _ptr(status, torch.int32, name="status"),
                                       _stream(stream)))


class Solver:
    """Owns one ucn_problem and the device buffers of its results."""

    def __init__(self, prob, precision=UCN_PREC_FP64, timeout_s=0.0, device="cuda", **overrides):
        import torch
        self.prob = prob
        self.precision = precision
        desc, keep = make_desc(prob, precision, timeout_s, **overrides)
        self.handle = ucn_problem_create(desc)
        del keep
        self.B = len(prob.N)
        self.nx, self.nu = int(prob.nx), int(prob.nu)
        self.tx, self.tu = ucn_total_x(self.handle), ucn_total_u(self.handle)
        dev = torch.device(device)
        self.x_out = torch.zeros(self.tx, self.nx, dtype=torch.float64, device=dev)
        self.u_out = torch.zeros(self.tu, self.nu, dtype=torch.float64, device=dev)
        self.stats = torch.zeros(self.B * 128, dtype=torch.uint8, device=dev)
        self.status = torch.zeros(self.B, dtype=torch.int32, device=dev)
        self.device = dev

    def close(self):
        if self.handle is not None:
            ucn_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tensor(self, a, dtype=None):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device=self.device)

    def scp_solve(self, x0=None, u0=None, stream=None, state=None):
        """Launch the fused SCP kernel (from the ADMM ``state`` when given: a
        warm start); returns the output tensors (not synchronised)."""
        x0 = self.tensor(self.prob.xguess) if x0 is None else x0
        u0 = self.tensor(self.prob.uguess) if u0 is None else u0
        if state is None:
            ucn_scp_solve(self.handle, x0, u0, self.x_out, self.u_out, self.stats, self.status, stream)
        else:
            ucn_scp_solve_warm(self.handle, x0, u0, state, self.x_out, self.u_out, self.stats, self.status, stream)
        return self.x_out, self.u_out

    def mpc_shift(self, x=None, u=None, stream=None):
        """Receding-horizon step from the last solution; returns the next
        guesses (x, u) as new device tensors."""
        import torch
        x = self.x_out if x is None else x
        u = self.u_out if u is None else u
        xg, ug = torch.empty_like(x), torch.empty_like(u)
        ucn_mpc_shift(self.handle, x, u, xg, ug, stream)
        return xg, ug

    def stats_host(self):
        return np.frombuffer(self.stats.cpu().numpy().tobytes(), dtype=STATS_DTYPE)

    def linearize(self, xbar, ubar, stream=None):
        import torch
        A = torch.empty(self.tu, self.nx, self.nx, dtype=torch.float64, device=self.device)
        B = torch.empty(self.tu, self.nx, self.nu, dtype=torch.float64, device=self.device)
        d = torch.empty(self.tu, self.nx, dtype=torch.float64, device=self.device)
        ucn_linearize(self.handle, xbar, ubar, A, B, d, stream)
        return A, B, d

    def admm_solve(self, xbar, ubar, A, B, d, radius, iters, warm=False, stream=None):
        import torch
        xhat = torch.empty(self.tx, self.nx, dtype=torch.float64, device=self.device)
        uhat = torch.empty(self.tu, self.nu, dtype=torch.float64, device=self.device)
        res = torch.empty(self.B, 2, dtype=torch.float64, device=self.device)
        status = torch.empty(self.B, dtype=torch.int32, device=self.device)
        ucn_admm_solve(self.handle, xbar, ubar, A, B, d, radius, iters, 1 if warm else 0, xhat, uhat, res, status, stream)
        return xhat, uhat, res, status

    def state_export(self, stream=None):
        import torch
        out = torch.empty(ucn_state_size(self.handle), dtype=torch.float64, device=self.device)
        ucn_state_export(self.handle, out, stream)
        return out
