"""Serving: continuous batching of SCP solves (binding of the ucn_serve_* ABI
and a host scheduling loop for request streams).

Requests are admitted into the server's slots as they arrive (while slots and
the HBM budget allow), every pump launches the admitted ones on a free lane
(stream) while earlier launches are still running, and finished results are
collected by non-blocking polls.  With the device-resident loop on
(Server.loop_start) a persistent kernel claims each request as it is submitted
instead, and pump only relaunches that kernel after an idle end.  Latency is
arrival -> result collected.
"""
from __future__ import annotations

import ctypes as C
import time
from collections import deque

import numpy as np

from . import ucn

_dp = C.POINTER(C.c_double)
_up = C.POINTER(C.c_ubyte)


class ServeConfig(C.Structure):
    _fields_ = [("model", C.c_int), ("precision", C.c_int), ("max_slots", C.c_int), ("max_horizon", C.c_int),
                ("max_obs", C.c_int), ("lanes", C.c_int), ("kept", C.c_int), ("hbm_budget_bytes", C.c_double),
                ("rho_eq", C.c_double), ("rho_dyn", C.c_double), ("rho_geo", C.c_double), ("rho_final", C.c_double),
                ("scp_iters", C.c_int), ("admm_iters", C.c_int), ("stop", C.c_int),
                ("tr_init", C.c_double), ("tr_min", C.c_double), ("tr_max", C.c_double), ("w_d", C.c_double),
                ("defect_tol", C.c_double), ("step_tol", C.c_double), ("timeout_s", C.c_double)]


class Request(C.Structure):
    _fields_ = [("horizon", C.c_int), ("n_obs", C.c_int), ("dt", C.c_double), ("model_params", _dp),
                ("Q_diag", _dp), ("x_ref", _dp), ("R_diag", _dp), ("u_ref", _dp), ("QN_diag", _dp), ("qN", _dp),
                ("x_lo", _dp), ("x_hi", _dp), ("u_lo", _dp), ("u_hi", _dp), ("x_init", _dp), ("x_target", _dp),
                ("term_mask", _up), ("obs_c", _dp), ("obs_r", _dp), ("sets", _dp),
                ("x_guess", _dp), ("u_guess", _dp), ("warm_ticket", C.c_ulonglong)]


class Result(C.Structure):
    _fields_ = [("stats", C.c_ubyte * 128), ("x", _dp), ("u", _dp), ("ticket", C.c_ulonglong),
                ("horizon", C.c_int), ("reserved", C.c_int)]


def _setup(L):
    if getattr(L, "_serve_ready", False):
        return L
    vp = C.c_void_p
    L.ucn_serve_create.argtypes = [C.POINTER(ServeConfig), C.POINTER(vp)]
    L.ucn_serve_create.restype = C.c_int
    L.ucn_serve_destroy.argtypes = [vp]
    L.ucn_serve_destroy.restype = None
    L.ucn_serve_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_ulonglong)]
    L.ucn_serve_submit.restype = C.c_int
    L.ucn_serve_pump.argtypes = [vp, C.POINTER(C.c_int)]
    L.ucn_serve_pump.restype = C.c_int
    L.ucn_serve_poll.argtypes = [vp, C.c_ulonglong, C.POINTER(Result)]
    L.ucn_serve_poll.restype = C.c_int
    L.ucn_serve_poll_any.argtypes = [vp, C.POINTER(Result)]
    L.ucn_serve_poll_any.restype = C.c_int
    L.ucn_serve_free_slots.argtypes = [vp]
    L.ucn_serve_free_slots.restype = C.c_int
    L.ucn_serve_loop_start.argtypes = [vp, C.c_int, C.c_double]
    L.ucn_serve_loop_start.restype = C.c_int
    L.ucn_serve_loop_stop.argtypes = [vp]
    L.ucn_serve_loop_stop.restype = C.c_int
    L.ucn_serve_loop_launches.argtypes = [vp]
    L.ucn_serve_loop_launches.restype = C.c_int
    L.ucn_serve_loop_capacity.argtypes = [vp]
    L.ucn_serve_loop_capacity.restype = C.c_int
    L._serve_ready = True
    return L


class Server:
    """One model / precision slot pool (ucn_serve_create)."""

    def __init__(self, model, precision, max_slots, max_horizon, max_obs=0, lanes=4, settings=None,
                 hbm_budget_bytes=0.0, kept=0, timeout_s=0.0):
        self.L = _setup(ucn.lib())
        s = settings or {}
        c = ServeConfig()
        c.model, c.precision, c.max_slots, c.max_horizon = model, precision, max_slots, max_horizon
        c.max_obs, c.lanes, c.kept, c.hbm_budget_bytes = max_obs, lanes, kept, float(hbm_budget_bytes)
        c.rho_eq, c.rho_dyn, c.rho_geo = float(s["rho_eq"]), float(s["rho_dyn"]), float(s["rho_geo"])
        c.rho_final = float(s.get("rho_final", 0.0))
        c.scp_iters, c.admm_iters, c.stop = int(s["scp_iters"]), int(s["admm_iters"]), int(s.get("stop", 0))
        c.tr_init, c.tr_min, c.tr_max, c.w_d = float(s["tr_init"]), float(s["tr_min"]), float(s["tr_max"]), float(s["w_d"])
        c.defect_tol, c.step_tol, c.timeout_s = float(s["defect_tol"]), float(s["step_tol"]), float(timeout_s)
        self.model, self.max_horizon = model, max_horizon
        self.nx, self.nu = {1: (12, 4), 2: (7, 3), 3: (13, 4), 4: (14, 3)}[model]
        self.h = C.c_void_p()
        rc = self.L.ucn_serve_create(C.byref(c), C.byref(self.h))
        if rc != ucn.UCN_OK:
            raise ucn.UcnError(rc, ucn.ucn_last_error())

    def close(self):
        if self.h is not None and self.h.value:
            self.L.ucn_serve_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prob, b=0, x_guess=None, u_guess=None, warm_ticket=0):
        """Returns (status, ticket).  Without a guess: warm start from `warm_ticket`
        if given, else the problem's own initial guess."""
        keep = []

        def d(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp)

        N = int(prob.N[b])
        r = Request()
        r.horizon, r.dt = N, float(prob.dt[b])
        r.n_obs = int(prob.nobs[b]) if prob.model in (1, 3) else 0
        r.model_params = d(prob.params[b])
        r.Q_diag, r.x_ref, r.R_diag, r.u_ref = d(prob.Qd[b]), d(prob.xref[b]), d(prob.Rd[b]), d(prob.uref[b])
        r.QN_diag, r.qN = d(prob.QNd[b]), d(prob.qN[b])
        r.x_lo, r.x_hi, r.u_lo, r.u_hi = d(prob.xlo[b]), d(prob.xhi[b]), d(prob.ulo[b]), d(prob.uhi[b])
        r.x_init, r.x_target = d(prob.xinit[b]), d(prob.xtarget[b])
        tm = np.ascontiguousarray(prob.tmask[b], dtype=np.uint8); keep.append(tm)
        r.term_mask = tm.ctypes.data_as(_up)
        if r.n_obs > 0:
            r.obs_c, r.obs_r = d(prob.obs_c[b, :r.n_obs]), d(prob.obs_r[b, :r.n_obs])
        r.sets = d(prob.sets[b])
        if warm_ticket:
            r.warm_ticket = int(warm_ticket)
        else:
            xo, uo = prob.xoff[b], prob.uoff[b]
            xg = prob.xguess[xo:xo + N + 1] if x_guess is None else x_guess
            ug = prob.uguess[uo:uo + N] if u_guess is None else u_guess
            r.x_guess, r.u_guess = d(xg), d(ug)
        t = C.c_ulonglong(0)
        rc = self.L.ucn_serve_submit(self.h, C.byref(r), C.byref(t))
        if rc not in (ucn.UCN_OK, ucn.UCN_EBUSY):
            raise ucn.UcnError(rc, ucn.ucn_last_error())
        return rc, int(t.value)

    def pump(self):
        n = C.c_int(0)
        rc = self.L.ucn_serve_pump(self.h, C.byref(n))
        if rc not in (ucn.UCN_OK, ucn.UCN_EBUSY):
            raise ucn.UcnError(rc, ucn.ucn_last_error())
        return rc, int(n.value)

    def poll(self, ticket, horizon=None, trajectories=True):
        """(status, result dict or None); status UCN_EBUSY while not finished."""
        res = Result()
        x = u = None
        if trajectories and horizon is not None:
            x = np.zeros((horizon + 1, self.nx)); u = np.zeros((horizon, self.nu))
            res.x, res.u = x.ctypes.data_as(_dp), u.ctypes.data_as(_dp)
        rc = self.L.ucn_serve_poll(self.h, C.c_ulonglong(ticket), C.byref(res))
        if rc == ucn.UCN_EBUSY:
            return rc, None
        if rc != ucn.UCN_OK:
            raise ucn.UcnError(rc, ucn.ucn_last_error())
        st = np.frombuffer(bytes(res.stats), dtype=ucn.STATS_DTYPE)[0]
        return rc, {"ticket": int(res.ticket), "horizon": int(res.horizon), "stats": st, "x": x, "u": u}

    def poll_any(self, trajectories=False):
        """(status, ticket, result dict) of some finished request; status
        UCN_EBUSY (and None, None) when none has finished.  The dict holds
        "stats", and "x", "u" when `trajectories`."""
        res = Result()
        x = u = None
        if trajectories:
            x = np.zeros((self.max_horizon + 1, self.nx)); u = np.zeros((self.max_horizon, self.nu))
            res.x, res.u = x.ctypes.data_as(_dp), u.ctypes.data_as(_dp)
        rc = self.L.ucn_serve_poll_any(self.h, C.byref(res))
        if rc == ucn.UCN_EBUSY:
            return rc, None, None
        if rc != ucn.UCN_OK:
            raise ucn.UcnError(rc, ucn.ucn_last_error())
        out = {"stats": np.frombuffer(bytes(res.stats), dtype=ucn.STATS_DTYPE)[0]}
        if trajectories:
            N = int(res.horizon)
            out["x"], out["u"] = x[:N + 1].copy(), u[:N].copy()
        return rc, int(res.ticket), out

    def free_slots(self):
        return int(self.L.ucn_serve_free_slots(self.h))

    def loop_start(self, ctas=0, idle_s=1.0):
        """Switch to the device-resident request loop (ucn_serve_loop_start):
        from here on every submit is published to a persistent kernel whose
        CTAs claim and solve requests as they free up; pump only relaunches the
        loop after an idle end."""
        rc = self.L.ucn_serve_loop_start(self.h, int(ctas), float(idle_s))
        if rc != ucn.UCN_OK:
            raise ucn.UcnError(rc, ucn.ucn_last_error())

    def loop_stop(self):
        """Serve what is queued, end the loop kernel, back to pump launches."""
        rc = self.L.ucn_serve_loop_stop(self.h)
        if rc != ucn.UCN_OK:
            raise ucn.UcnError(rc, ucn.ucn_last_error())

    def loop_launches(self):
        return int(self.L.ucn_serve_loop_launches(self.h))

    def loop_capacity(self):
        """CTAs of this server's loop kernel that can be resident at once."""
        n = int(self.L.ucn_serve_loop_capacity(self.h))
        if n < 0:
            raise ucn.UcnError(ucn.UCN_EINVAL, ucn.ucn_last_error())
        return n


def horizon_route(buckets):
    """A route for run_stream over servers keyed (model, max_horizon): each
    request to its model's server with the smallest max_horizon that holds it
    (a server's CTA size and node layout follow its max_horizon, so short
    requests run in small CTAs with their records in shared memory)."""
    def route(p):
        N = int(p.N[0])
        return (p.model, min(h for h in buckets[p.model] if h >= N))
    return route


def server_name(key):
    """A server key as text: "1" for a model, "1/40" for (model, max_horizon)."""
    return "/".join(str(v) for v in key) if isinstance(key, tuple) else str(key)


def run_stream(stream, servers, max_inflight=None, time_scale=1.0, route=None):
    """Replay a request stream [(arrival_s, Problem)] against `servers` in real
    time: a dict key -> Server, each request going to servers[route(request)]
    (default key: the request's model).  max_inflight=1 gives the one-at-a-time
    (per-request) path.  Returns latencies and throughput (also per model), and
    per server the number of solves and their mean device time (start to end of
    the solve's CTA) in solve_ms_by_server, and how many ran at once
    (device_by_server)."""
    route = route or (lambda p: p.model)
    pending = deque(sorted(stream, key=lambda r: r[0]))
    waiting = {m: deque() for m in servers}     # arrived, not yet admitted, per server (FIFO)
    inflight = {}
    lat, defects, models = [], [], []
    busy = {m: [] for m in servers}     # device time of each solve (its CTA's start to end), per server
    n = len(pending)
    t0 = time.perf_counter()
    while len(lat) < n:
        now = (time.perf_counter() - t0) / time_scale
        while pending and pending[0][0] <= now:
            arr, p = pending.popleft()
            waiting[route(p)].append((arr, p))
        for m, q in waiting.items():
            # admit in arrival order per server; a full server does not hold up the others
            while q and (max_inflight is None or len(inflight) < max_inflight):
                arr, p = q[0]
                rc, ticket = servers[m].submit(p)
                if rc == ucn.UCN_EBUSY:
                    break
                q.popleft()
                inflight[(m, ticket)] = (arr, p.model)
        for srv in servers.values():
            srv.pump()
        for key, srv in servers.items():
            # every request finished since the last pass (one call each)
            while True:
                rc, ticket, res = srv.poll_any()
                if rc != ucn.UCN_OK:
                    break
                arr, model = inflight.pop((key, ticket))
                lat.append((time.perf_counter() - t0) / time_scale - arr)
                st = res["stats"]
                defects.append(float(st["defect"]))
                models.append(model)
                busy[key].append((int(st["t_start_ns"]), int(st["t_end_ns"])))
    elapsed = time.perf_counter() - t0
    lat = np.array(lat)
    d = np.array(defects)
    models = np.array(models)
    out = {"completed": n, "elapsed_s": elapsed, "solves_per_s": float(np.sum(d <= 1e-5)) / elapsed,
           "requests_per_s": n / elapsed, "pass_rate": float(np.mean(d <= 1e-5)),
           "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99))}
    for m in np.unique(models):
        lm = lat[models == m]
        out["model%d" % m] = {"requests": int(lm.size), "p50_ms": 1e3 * float(np.percentile(lm, 50)),
                              "p99_ms": 1e3 * float(np.percentile(lm, 99))}
    out["solve_ms_by_server"] = {server_name(k): [len(v), 1e-6 * float(np.mean([e - b for b, e in v]))]
                                 for k, v in busy.items() if v}
    out["device_by_server"] = {server_name(k): device_use(v) for k, v in busy.items() if v}
    return out


def device_use(spans):
    """Solves of one server on the device, from their (start, end) timestamps in
    ns: the most that ran at once, and the device time they took in all over the
    span from the first start to the last end (mean solves running at once)."""
    ev = sorted([(b, 1) for b, _ in spans] + [(e, -1) for _, e in spans])
    run = most = 0
    for _, d in ev:
        run += d
        most = max(most, run)
    first, last = min(b for b, _ in spans), max(e for _, e in spans)
    total = float(sum(e - b for b, e in spans))
    return {"max_running": most, "span_s": 1e-9 * (last - first), "mean_running": total / max(last - first, 1)}
