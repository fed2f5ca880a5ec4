"""Seeded synthetic problem generators.

This module serves both the FP64 CPU oracle (``oracle/``) and the CUDA path
(``paper_2603_10711_gb300``).  It holds input data only -- problem constants,
random draws, initial guesses -- and none of the method's arithmetic: no
dynamics, no linearisation, no ADMM, no projection.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
2014): value = mix(seed * G + stream * K + index), with the published
finaliser ``mix``.  A draw is therefore a pure function of
(seed, stream, index); nothing depends on call order.

Workloads (shapes follow the paper's experiments, Sec. IV):

* ``quad_path``   -- quadrotor obstacle avoidance, obstacles placed along the
  straight start-goal path (one instance: the single-trajectory problem).
* ``mars_batch``  -- 3-DOF Mars powered descent, a batch of dispersed initial
  states (the paper's Monte-Carlo batch, Sec. IV-B).
* ``quad_box``    -- batched quadrotor planning with uneven horizons and
  obstacle counts in a 10 x 10 x 3 m box.
* ``double_integrator`` -- small linear test problems used by the oracle pins.

Units.  The quadrotor is in SI units.  The Mars problem is stored in
non-dimensional units (length 1000 m, time 10 s, mass 1905 kg), as the
paper's own Mars model is (Sec. IV-B); ``MARS_UNITS`` converts back.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict

import numpy as np

MODEL_QUAD12 = 1
MODEL_MARS7 = 2
MODEL_QUAT13 = 3
MODEL_MARS14 = 4
SET_PARAMS = 8          # set parameters per instance (thrust bounds, cone tangents, ...)

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAMK = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele et al. 2014), vectorised over uint64."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of mix(seed*G + stream*K + index)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * _GOLDEN + np.uint64(stream) * _STREAMK + idx)
    z = _mix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def U(seed, stream, index, lo, hi):
    """Uniform in [lo, hi) from counter ``index`` of ``stream``."""
    return lo + (hi - lo) * uniform(seed, stream, index)


@dataclasses.dataclass
class Problem:
    """A batch of B discrete optimal-control problems (the OCP of Eq. (1)).

    Trajectory arrays are packed per node: instance b owns state nodes
    ``xoff[b] .. xoff[b]+N[b]`` and control nodes ``uoff[b] .. uoff[b]+N[b]-1``.
    """

    model: int
    nx: int
    nu: int
    N: np.ndarray          # int32 [B]   horizon
    dt: np.ndarray         # f64 [B]     RK4 step
    params: np.ndarray     # f64 [B,8]   model constants (see model docs)
    Qd: np.ndarray         # f64 [B,nx]  running state weight (diagonal)
    xref: np.ndarray       # f64 [B,nx]
    Rd: np.ndarray         # f64 [B,nu]
    uref: np.ndarray       # f64 [B,nu]
    QNd: np.ndarray        # f64 [B,nx]  terminal weight (diagonal)
    qN: np.ndarray         # f64 [B,nx]  extra linear terminal term
    xlo: np.ndarray        # f64 [B,nx]  state box
    xhi: np.ndarray
    ulo: np.ndarray        # f64 [B,nu]  control box
    uhi: np.ndarray
    xinit: np.ndarray      # f64 [B,nx]
    xtarget: np.ndarray    # f64 [B,nx]
    tmask: np.ndarray      # u8  [B,nx]  selection S of the terminal constraint
    nobs: np.ndarray       # int32 [B]
    obs_c: np.ndarray      # f64 [B,max_obs,3]
    obs_r: np.ndarray      # f64 [B,max_obs]
    sets: np.ndarray       # f64 [B,4]   thrust_min, thrust_max, tan(glide half-angle), unused (<=0: off)
    xguess: np.ndarray     # f64 [sum(N+1), nx] initial nominal
    uguess: np.ndarray     # f64 [sum(N), nu]
    settings: Dict[str, float]

    @property
    def batch(self) -> int:
        return int(self.N.shape[0])

    @property
    def max_obs(self) -> int:
        return int(self.obs_r.shape[1])

    @property
    def xoff(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N.astype(np.int64) + 1)[:-1]]).astype(np.int64)

    @property
    def uoff(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.N.astype(np.int64))[:-1]]).astype(np.int64)

    @property
    def total_x(self) -> int:
        return int(np.sum(self.N.astype(np.int64) + 1))

    @property
    def total_u(self) -> int:
        return int(np.sum(self.N.astype(np.int64)))

    def subset(self, idx) -> "Problem":
        """The instances ``idx`` as a problem of their own (same settings)."""
        idx = np.asarray(idx, dtype=np.int64)
        xo, uo, N = self.xoff, self.uoff, self.N
        xs = np.concatenate([self.xguess[xo[b]:xo[b] + N[b] + 1] for b in idx])
        us = np.concatenate([self.uguess[uo[b]:uo[b] + N[b]] for b in idx])
        f = {}
        for fld in dataclasses.fields(self):
            v = getattr(self, fld.name)
            if fld.name in ("model", "nx", "nu", "settings"):
                f[fld.name] = v if fld.name != "settings" else dict(v)
            elif fld.name == "xguess":
                f[fld.name] = xs
            elif fld.name == "uguess":
                f[fld.name] = us
            else:
                f[fld.name] = np.ascontiguousarray(v[idx])
        return Problem(**f)


DEFAULT_SETTINGS = dict(
    rho_eq=1.0, rho_dyn=1.0, rho_geo=1.0, rho_final=0.0,
    scp_iters=15, admm_iters=200, stop=0,
    tr_init=1.0, tr_min=1e-6, tr_max=10.0,
    w_d=1e3, defect_tol=1e-5, step_tol=1e-6, vc_weight=0.0,
)

# ---------------------------------------------------------------- quadrotor
QUAD_MASS = 1.0
QUAD_J = (0.01, 0.01, 0.02)
QUAD_ARM = 0.2
QUAD_KM = 0.01   # yaw moment per unit rotor thrust [m]; not given, proposed
QUAD_G = 9.81
QUAD_UMAX = 5.0


def _quad_params(B, mass=None, cd=None):
    p = np.zeros((B, 8))
    p[:, 0] = QUAD_MASS if mass is None else mass
    p[:, 1:4] = QUAD_J
    p[:, 4] = QUAD_ARM
    p[:, 5] = QUAD_KM
    p[:, 6] = 0.0 if cd is None else cd
    p[:, 7] = QUAD_G
    return p


def _quad_common(B, N, dt, start, goal, obs_c, obs_r, nobs, settings, mass=None, cd=None):
    nx, nu = 12, 4
    params = _quad_params(B, mass, cd)
    hover = params[:, 0] * QUAD_G / 4.0
    xinit = np.zeros((B, nx)); xinit[:, 0:3] = start
    xtarget = np.zeros((B, nx)); xtarget[:, 0:3] = goal
    tmask = np.zeros((B, nx), np.uint8); tmask[:, 0:6] = 1   # position + velocity
    xref = xtarget.copy()
    uref = np.repeat(hover[:, None], nu, axis=1)
    xs, us = [], []
    for b in range(B):
        s = np.arange(N[b] + 1)[:, None] / N[b]
        xb = np.zeros((N[b] + 1, nx))
        xb[:, 0:3] = (1 - s) * start[b] + s * goal[b]
        xs.append(xb)
        us.append(np.full((N[b], nu), hover[b]))
    st = dict(DEFAULT_SETTINGS); st.update(settings)
    return Problem(
        model=MODEL_QUAD12, nx=nx, nu=nu, N=np.asarray(N, np.int32), dt=np.full(B, dt),
        params=params, Qd=np.ones((B, nx)), xref=xref, Rd=np.full((B, nu), 0.1), uref=uref,
        QNd=np.ones((B, nx)), qN=np.zeros((B, nx)),
        xlo=np.full((B, nx), -np.inf), xhi=np.full((B, nx), np.inf),
        ulo=np.zeros((B, nu)), uhi=np.full((B, nu), QUAD_UMAX),
        xinit=xinit, xtarget=xtarget, tmask=tmask,
        nobs=np.asarray(nobs, np.int32), obs_c=obs_c, obs_r=obs_r, sets=np.zeros((B, SET_PARAMS)),
        xguess=np.concatenate(xs), uguess=np.concatenate(us), settings=st)


def quad_path(B=1, seed=0, N=50, dt=0.05, n_obs=5, settings=None) -> Problem:
    """Quadrotor obstacle avoidance (the paper's quadrotor task, Sec. IV-A).

    Start at the origin hovering; goal ~ U([4,6]x[-1,1]x[0.5,1.5]) m;
    ``n_obs`` spheres with centre = start + s (goal - start) + U[-0.5,0.5]^3,
    s ~ U[0.2,0.8], radius ~ U[0.3,0.6] m.  A sphere that would contain the
    start or the goal (with 0.1 m margin) is redrawn from the next counters.
    Controls: four rotor thrusts boxed to [0, 5] N; Q = I, R = 0.1 I.
    """
    goal = np.stack([U(seed, 1, np.arange(B) * 8 + k, lo, hi)
                     for k, (lo, hi) in enumerate([(4, 6), (-1, 1), (0.5, 1.5)])], axis=1)
    start = np.zeros((B, 3))
    obs_c = np.zeros((B, n_obs, 3)); obs_r = np.zeros((B, n_obs))
    for b in range(B):
        for j in range(n_obs):
            for attempt in range(1000):
                base = (b * 4096 + j * 64 + attempt) * 8
                s = U(seed, 2, base, 0.2, 0.8)
                off = U(seed, 3, base + np.arange(3), -0.5, 0.5)
                r = U(seed, 4, base, 0.3, 0.6)
                c = start[b] + s * (goal[b] - start[b]) + off
                if (np.linalg.norm(c - start[b]) > r + 0.1 and np.linalg.norm(c - goal[b]) > r + 0.1):
                    break
            obs_c[b, j] = c; obs_r[b, j] = r
    return _quad_common(B, np.full(B, N), dt, start, goal, obs_c, obs_r, np.full(B, n_obs),
                        settings or {})


QUAT_TMAX, QUAT_TAUMAX = 20.0, 5.0     # N, N m


def quat_study(B=1, seed=5, N=50, tf=6.0, n_obs=3, rho0=1.0, rho_final=1e3, scp_iters=20, admm_iters=100,
               settings=None) -> Problem:
    """The paper's 13-state quadrotor parameter study (Sec. IV-A2): a 6 s flight
    (N = 50) from hover at (-5, -5, 2) m to (5, 5, 2) m with the terminal
    position and zero velocity enforced; three spheres of radius U[1.2, 1.5] m
    on the direct path (centres at s = 1/4, 1/2, 3/4 of it, s jittered by
    U[-0.05, 0.05], offset U[-0.6, 0.6] m across and U[-0.3, 0.3] m in height);
    thrust in [0, 20] N, torques in [-5, 5] N m; m = 1 kg, g = 9.81, J as the
    12-state model.  Cost Q = I about the goal state (identity attitude), R =
    0.1 I about hover.  All three penalties start at rho0 and rise
    geometrically to rho_final over the scp_iters SCP iterations (fixed count).
    """
    nx, nu = 13, 4
    start = np.array([-5.0, -5.0, 2.0]); goal = np.array([5.0, 5.0, 2.0])
    d = goal - start
    across = np.array([-d[1], d[0], 0.0]) / np.linalg.norm(d[:2])
    obs_c = np.zeros((B, n_obs, 3)); obs_r = np.zeros((B, n_obs))
    for b in range(B):
        for j in range(n_obs):
            base = (b * 64 + j) * 8
            sj = (j + 1) / (n_obs + 1) + U(seed, 60, base, -0.05, 0.05)
            c = start + sj * d + U(seed, 61, base, -0.6, 0.6) * across + np.array([0.0, 0.0, U(seed, 62, base, -0.3, 0.3)])
            obs_c[b, j] = c
            obs_r[b, j] = U(seed, 63, base, 1.2, 1.5)
    params = _quad_params(B)
    hover = params[:, 0] * QUAD_G
    xinit = np.zeros((B, nx)); xinit[:, 0:3] = start; xinit[:, 6] = 1.0
    xtarget = np.zeros((B, nx)); xtarget[:, 0:3] = goal; xtarget[:, 6] = 1.0
    tmask = np.zeros((B, nx), np.uint8); tmask[:, 0:6] = 1
    uref = np.zeros((B, nu)); uref[:, 0] = hover
    s_ = np.arange(N + 1)[:, None] / N
    xs, us = [], []
    for b in range(B):
        xb = np.zeros((N + 1, nx)); xb[:, 0:3] = (1 - s_) * start + s_ * goal; xb[:, 6] = 1.0
        xs.append(xb)
        ub = np.zeros((N, nu)); ub[:, 0] = hover[b]
        us.append(ub)
    st = dict(DEFAULT_SETTINGS)
    st.update(dict(rho_eq=rho0, rho_dyn=rho0, rho_geo=rho0, rho_final=rho_final, scp_iters=scp_iters,
                   admm_iters=admm_iters, stop=0))
    st.update(settings or {})
    return Problem(
        model=MODEL_QUAT13, nx=nx, nu=nu, N=np.full(B, N, np.int32), dt=np.full(B, tf / N),
        params=params, Qd=np.ones((B, nx)), xref=xtarget.copy(), Rd=np.full((B, nu), 0.1), uref=uref,
        QNd=np.ones((B, nx)), qN=np.zeros((B, nx)),
        xlo=np.full((B, nx), -np.inf), xhi=np.full((B, nx), np.inf),
        ulo=np.tile([0.0, -QUAT_TAUMAX, -QUAT_TAUMAX, -QUAT_TAUMAX], (B, 1)),
        uhi=np.tile([QUAT_TMAX, QUAT_TAUMAX, QUAT_TAUMAX, QUAT_TAUMAX], (B, 1)),
        xinit=xinit, xtarget=xtarget, tmask=tmask,
        nobs=np.full(B, n_obs, np.int32), obs_c=obs_c, obs_r=obs_r, sets=np.zeros((B, SET_PARAMS)),
        xguess=np.concatenate(xs), uguess=np.concatenate(us), settings=st)


def quad_box(B=4096, seed=2, N_range=(40, 120), obs_range=(10, 30), dt=0.05,
             settings=None) -> Problem:
    """Batched quadrotor planning with uneven sizes in a 10 x 10 x 3 m box.

    N_b ~ U{40..120}; 10..30 spheres per instance with radius ~ U[0.2,0.8] m
    and centres uniform in the box; start and goal uniform in the box and at
    least 0.2 m clear of every sphere (redrawn otherwise).  Settings: rho = 10,
    200 ADMM iterations per SCP iteration, cap 40, stop at defect <= 1e-5.
    """
    lo = np.array([0.0, 0.0, 0.0]); hi = np.array([10.0, 10.0, 3.0])
    Ns = (N_range[0] + np.floor(uniform(seed, 10, np.arange(B)) * (N_range[1] - N_range[0] + 1))).astype(np.int32)
    nobs = (obs_range[0] + np.floor(uniform(seed, 11, np.arange(B)) * (obs_range[1] - obs_range[0] + 1))).astype(np.int32)
    mo = int(obs_range[1])
    obs_c = np.zeros((B, mo, 3)); obs_r = np.zeros((B, mo))
    start = np.zeros((B, 3)); goal = np.zeros((B, 3))
    for b in range(B):
        for j in range(nobs[b]):
            base = (b * 64 + j) * 8
            obs_c[b, j] = U(seed, 12, base + np.arange(3), lo, hi)
            obs_r[b, j] = U(seed, 13, base, 0.2, 0.8)
        for k, arr in ((0, start), (1, goal)):
            for attempt in range(10000):
                base = ((b * 2 + k) * 10000 + attempt) * 4
                p = U(seed, 14, base + np.arange(3), lo + 0.5, hi - 0.5)
                d = np.linalg.norm(obs_c[b, :nobs[b]] - p, axis=1) - obs_r[b, :nobs[b]]
                if nobs[b] == 0 or d.min() > 0.2:
                    break
            arr[b] = p
    st = dict(rho_eq=10.0, rho_dyn=10.0, rho_geo=10.0, scp_iters=40, admm_iters=200, stop=1, step_tol=1.0)
    st.update(settings or {})
    return _quad_common(B, Ns, dt, start, goal, obs_c, obs_r, nobs, st)


# ---------------------------------------------------------------- Mars 3-DOF
MARS_UNITS = dict(length=1000.0, time=10.0, mass=1905.0)   # m, s, kg
MARS_G = 3.71            # m/s^2
MARS_ISP = 225.0         # s
MARS_G0 = 9.80665        # m/s^2 (standard gravity in the rocket equation)
MARS_TMIN, MARS_TMAX = 4800.0, 19200.0   # N
MARS_WET, MARS_DRY = 1905.0, 1505.0      # kg; dry mass not given, proposed
MARS_GLIDE_DEG = 86.0    # half-angle of the glide-slope cone, from vertical


def mars_units():
    L, T, M = MARS_UNITS["length"], MARS_UNITS["time"], MARS_UNITS["mass"]
    return dict(L=L, T=T, M=M, V=L / T, A=L / T ** 2, F=M * L / T ** 2)


def mars_batch(B=1024, seed=1, N=100, tf=60.0, settings=None) -> Problem:
    """Mars powered descent batch, 3-DOF (position, velocity, mass; Up-East-North).

    r0 ~ U([1500,2500]x[-500,500]^2) m, v0 ~ U([-80,-40]x[-20,20]^2) m/s,
    m0 = 1905 kg; |T| in [4.8, 19.2] kN; glide slope 86 deg; Isp = 225 s;
    g = 3.71 m/s^2; land at r = 0, v = 0; cost -m_N (fuel optimal).
    Stored non-dimensionally (``MARS_UNITS``).
    """
    u = mars_units()
    nx, nu = 7, 3
    r0 = np.stack([U(seed, 21, np.arange(B) * 8 + k, lo, hi) for k, (lo, hi) in
                   enumerate([(1500, 2500), (-500, 500), (-500, 500)])], axis=1) / u["L"]
    v0 = np.stack([U(seed, 22, np.arange(B) * 8 + k, lo, hi) for k, (lo, hi) in
                   enumerate([(-80, -40), (-20, 20), (-20, 20)])], axis=1) / u["V"]
    m0 = MARS_WET / u["M"]
    params = np.zeros((B, 8))
    params[:, 0] = MARS_G / u["A"]
    params[:, 1] = (1.0 / (MARS_ISP * MARS_G0)) * u["F"] * u["T"] / u["M"]
    xinit = np.zeros((B, nx)); xinit[:, 0:3] = r0; xinit[:, 3:6] = v0; xinit[:, 6] = m0
    xtarget = np.zeros((B, nx))
    tmask = np.zeros((B, nx), np.uint8); tmask[:, 0:6] = 1
    tmin, tmax = MARS_TMIN / u["F"], MARS_TMAX / u["F"]
    sets = np.zeros((B, SET_PARAMS)); sets[:, 0] = tmin; sets[:, 1] = tmax
    sets[:, 2] = math.tan(math.radians(MARS_GLIDE_DEG))
    xlo = np.full((B, nx), -np.inf); xhi = np.full((B, nx), np.inf)
    xlo[:, 6] = MARS_DRY / u["M"]; xhi[:, 6] = m0
    qN = np.zeros((B, nx)); qN[:, 6] = -1.0
    hover = m0 * params[:, 0]
    xs, us = [], []
    for b in range(B):
        s = np.arange(N + 1)[:, None] / N
        xb = np.zeros((N + 1, nx))
        xb[:, 0:6] = (1 - s) * xinit[b, 0:6]
        xb[:, 6] = m0
        xs.append(xb)
        ub = np.zeros((N, nu)); ub[:, 0] = hover[b]
        us.append(ub)
    st = dict(DEFAULT_SETTINGS)
    # Paper's geometric penalty schedule (Sec. IV-A: all three rho equal, raised
    # geometrically over the SCP iterations), here 1 -> 1e7 over a 60-iteration
    # cap with 40 ADMM iterations each (the least ADMM work of an oracle sweep at
    # which every instance passes, with the fuel of 1 -> 1e5 over 150 x 100); the
    # solve stops once the defect of an accepted candidate is <= 1e-5 (the step
    # test is switched off: step_tol = 1).
    st.update(dict(rho_eq=1.0, rho_dyn=1.0, rho_geo=1.0, rho_final=1e7, scp_iters=60,
                   admm_iters=40, stop=1, step_tol=1.0))
    st.update(settings or {})
    return Problem(
        model=MODEL_MARS7, nx=nx, nu=nu, N=np.full(B, N, np.int32), dt=np.full(B, tf / N / u["T"]),
        params=params, Qd=np.zeros((B, nx)), xref=np.zeros((B, nx)), Rd=np.zeros((B, nu)),
        uref=np.zeros((B, nu)), QNd=np.zeros((B, nx)), qN=qN,
        xlo=xlo, xhi=xhi, ulo=np.full((B, nu), -tmax), uhi=np.full((B, nu), tmax),
        xinit=xinit, xtarget=xtarget, tmask=tmask,
        nobs=np.zeros(B, np.int32), obs_c=np.zeros((B, 0, 3)), obs_r=np.zeros((B, 0)), sets=sets,
        xguess=np.concatenate(xs), uguess=np.concatenate(us), settings=st)


# ---------------------------------------------------------------- linear test QPs
def double_integrator(seed=0, N=3, nx=2, nu=1, dt=0.1):
    """Random small linear-quadratic data for the oracle's pins.

    Returns per-node arrays A[N,nx,nx], B[N,nx,nu], d[N,nx] (a perturbed
    discretised double integrator), SPD Q[N+1,nx,nx], R[N,nu,nu], cross
    terms M[N,nx,nu] small enough to keep the stage Hessians SPD, linear
    terms q, r and an initial state.
    """
    k = 0

    def draw(shape, lo=-1.0, hi=1.0):
        nonlocal k
        n = int(np.prod(shape))
        v = U(seed, 31, np.arange(k, k + n), lo, hi).reshape(shape)
        k += n
        return v

    A = np.zeros((N, nx, nx)); Bm = np.zeros((N, nx, nu))
    for i in range(N):
        A[i] = np.eye(nx) + 0.1 * draw((nx, nx))
        if nx >= 2:
            A[i, 0, 1] += dt
        Bm[i] = 0.5 * draw((nx, nu))
        Bm[i, -1, :] += dt
    d = 0.1 * draw((N, nx))
    Q = np.zeros((N + 1, nx, nx)); R = np.zeros((N, nu, nu)); M = np.zeros((N, nx, nu))
    for i in range(N + 1):
        G = draw((nx, nx)); Q[i] = G @ G.T / nx + 0.5 * np.eye(nx)
    for i in range(N):
        G = draw((nu, nu)); R[i] = G @ G.T / nu + 0.5 * np.eye(nu)
        M[i] = 0.1 * draw((nx, nu))
    q = draw((N + 1, nx)); r = draw((N, nu))
    x0 = draw((nx,))
    return dict(A=A, B=Bm, d=d, Q=Q, R=R, M=M, q=q, r=r, x0=x0, N=N, nx=nx, nu=nu)


# ---------------------------------------------------------------- serving stream
def serving_stream(n: int, rate: float, seed: int = 4, quad_share: float = 0.7):
    """A Poisson request stream mixing quadrotor and Mars-descent solves.

    Arrival gaps ~ Exp(rate) (inverse transform of the counter generator).
    70% quadrotor (N ~ U{30..120}, 5..30 obstacles in the 10 x 10 x 3 m box)
    and 30% Mars descent (N ~ U{50..200}, t_f = 60 s), each a one-instance
    Problem with its workload's solver settings.  Returns a list of
    (arrival_time_s, Problem)."""
    u_gap = uniform(seed, 41, np.arange(n))
    t = np.cumsum(-np.log1p(-u_gap) / rate)
    kind = uniform(seed, 42, np.arange(n)) < quad_share
    u_n = uniform(seed, 43, np.arange(n))
    u_o = uniform(seed, 44, np.arange(n))
    out = []
    for k in range(n):
        if kind[k]:
            N = 30 + int(u_n[k] * 91)
            no = 5 + int(u_o[k] * 26)
            p = quad_box(1, seed=1000 + k, N_range=(N, N), obs_range=(no, no))
        else:
            N = 50 + int(u_n[k] * 151)
            p = mars_batch(1, seed=5000 + k, N=N)
        out.append((float(t[k]), p))
    return out


# ---------------------------------------------------------------- scenario MPC
def scenario_mpc(P=256, K=16, seed=3, N=40, n_obs=8, dt=0.05, settings=None) -> Problem:
    """Scenario-based robust planning (the paper's robust MPC, Sec. IV-A):
    P problems x K scenarios.  Each problem draws start, goal and `n_obs`
    spheres in the 10 x 10 x 3 m box (like ``quad_box``); its K scenarios share
    them and differ in mass ~ U[0.9, 1.1] kg and linear drag ~ U[0, 0.2].
    Instances b = p*K + s; settings["group"] = K couples the scenarios of a
    problem through their first control.  As in receding-horizon control the
    goal is not a terminal equality (a 2 s horizon cannot always reach it):
    the terminal cost weighs position and velocity by 10 instead."""
    base = quad_box(P, seed=seed, N_range=(N, N), obs_range=(n_obs, n_obs), dt=dt)
    idx = np.repeat(np.arange(P), K)
    prob = base.subset(idx)
    mass = U(seed, 51, np.arange(P * K), 0.9, 1.1)
    cd = U(seed, 52, np.arange(P * K), 0.0, 0.2)
    prob.params[:, 0] = mass
    prob.params[:, 6] = cd
    prob.tmask[:] = 0
    prob.QNd[:, :6] = 10.0
    hover = mass * QUAD_G / 4.0
    prob.uref[:] = hover[:, None]
    for b in range(P * K):
        uo = prob.uoff[b]
        prob.uguess[uo:uo + N] = hover[b]
    st = dict(DEFAULT_SETTINGS)
    st.update(dict(rho_eq=10.0, rho_dyn=10.0, rho_geo=10.0, scp_iters=40, admm_iters=200, stop=1, step_tol=1.0,
                   group=K))
    st.update(settings or {})
    prob.settings = st
    return prob


# ---------------------------------------------------------------- Mars 6-DOF
MARS6_ALPHA, MARS6_G = 0.1, 1.0                  # non-dimensional
MARS6_J = (0.0168, 0.168, 0.168)                 # diagonal inertia (not given; proposed)
MARS6_LEVER = 1.0                                # thrust applied at -l e_x in the body (proposed)


def mars6_batch(B=1000, seed=7, N=30, tf=5.0, settings=None) -> Problem:
    """The paper's 6-DOF Mars landing (Sec. IV-B1) as a Monte-Carlo batch
    (Sec. IV-B2), non-dimensional units: state (m, r Up-East-North, v, q, omega),
    control = body-frame thrust; m' = -0.1 |T|, g = 1 along -Up; mass in
    [0.75, 2.0]; |T| in [0.5, 3.0]; gimbal <= 10 deg from the body x axis; glide
    slope 10 deg above the horizon; tilt <= 20 deg from Up; |omega| <= 30 deg per
    unit time; horizon 5.0 in N = 30 steps.  Nominal start m = 2, r = (2, 1, 0),
    v = (-1, 0.2, 0), upright, at rest; every component perturbed by U[-0.05,
    0.05] (mass downward only; quaternion renormalised); touchdown at r = 0 with
    v = (-0.1, 0, 0) and the body upright (roll about the thrust axis free);
    cost = -m_N (fuel).
    """
    nx, nu = 14, 3
    x0n = np.array([2.0, 2.0, 1.0, 0.0, -1.0, 0.2, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    pert = np.stack([U(seed, 70 + k, np.arange(B), -0.05, 0.05) for k in range(nx)], axis=1)
    pert[:, 0] = -np.abs(pert[:, 0])
    xinit = x0n[None, :] + pert
    xinit[:, 7:11] /= np.linalg.norm(xinit[:, 7:11], axis=1, keepdims=True)
    xtarget = np.zeros((B, nx)); xtarget[:, 4] = -0.1; xtarget[:, 7] = 1.0
    # touchdown: position, velocity and an upright body (qy = qz = 0); the roll
    # about the thrust axis and the rates stay free (no torque acts about that axis)
    tmask = np.zeros((B, nx), np.uint8); tmask[:, 1:7] = 1; tmask[:, 9:11] = 1
    params = np.zeros((B, 8))
    params[:, 0] = MARS6_ALPHA; params[:, 1] = MARS6_G; params[:, 2:5] = MARS6_J; params[:, 5] = MARS6_LEVER
    sets = np.zeros((B, SET_PARAMS))
    sets[:, 0] = 0.5; sets[:, 1] = 3.0
    sets[:, 2] = math.tan(math.radians(90.0 - 10.0))       # glide slope: 10 deg above the horizon
    sets[:, 3] = math.tan(math.radians(10.0))              # gimbal
    sets[:, 4] = math.sin(math.radians(20.0) / 2)          # tilt: |(qy, qz)| <= sin(theta / 2)
    sets[:, 5] = math.radians(30.0)                        # body rate
    xlo = np.full((B, nx), -np.inf); xhi = np.full((B, nx), np.inf)
    xlo[:, 0] = 0.75; xhi[:, 0] = 2.0
    qN = np.zeros((B, nx)); qN[:, 0] = -1.0
    s_ = np.arange(N + 1)[:, None] / N
    xs, us = [], []
    for b in range(B):
        xb = (1 - s_) * xinit[b] + s_ * xtarget[b]
        xb[:, 0] = xinit[b, 0]
        xb[:, 7:11] = np.array([1.0, 0, 0, 0]); xb[0, 7:11] = xinit[b, 7:11]
        xb[:, 11:14] = 0.0; xb[0, 11:14] = xinit[b, 11:14]
        xs.append(xb)
        ub = np.zeros((N, nu)); ub[:, 0] = xinit[b, 0] * MARS6_G
        us.append(ub)
    st = dict(DEFAULT_SETTINGS)
    st.update(dict(rho_eq=1.0, rho_dyn=1.0, rho_geo=1.0, rho_final=1e5, scp_iters=150, admm_iters=100, stop=1,
                   step_tol=1.0))
    st.update(settings or {})
    return Problem(
        model=MODEL_MARS14, nx=nx, nu=nu, N=np.full(B, N, np.int32), dt=np.full(B, tf / N), params=params,
        Qd=np.zeros((B, nx)), xref=np.zeros((B, nx)), Rd=np.zeros((B, nu)), uref=np.zeros((B, nu)),
        QNd=np.zeros((B, nx)), qN=qN, xlo=xlo, xhi=xhi,
        ulo=np.full((B, nu), -np.inf), uhi=np.full((B, nu), np.inf),
        xinit=xinit, xtarget=xtarget, tmask=tmask,
        nobs=np.zeros(B, np.int32), obs_c=np.zeros((B, 0, 3)), obs_r=np.zeros((B, 0)), sets=sets,
        xguess=np.concatenate(xs), uguess=np.concatenate(us), settings=st)
