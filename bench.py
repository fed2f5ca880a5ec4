"""Benchmark: SCP solves/s at max nonlinear defect <= 1e-5 on one GB300.

Workload: the Mars powered-descent batch (1024 instances, N = 100, 3-DOF,
|T| in [4.8, 19.2] kN, glide slope 86 deg), solved by the fused persistent
SCP kernel in the FP32 + refinement path (ADMM in FP32; nominal, rollout and
merits in double-float; acceptance test, returned trajectory and its defect
in FP64).  One step = one ucn_scp_solve over the whole batch (two launches of
the fused kernel: a first round of three CTAs per SM, then the rest).  `value`
counts only solves whose returned trajectory has max defect <= 1e-5 (an FP64
RK4 defect of the returned doubles, computed by the kernel; the parity leg
recomputes it with the oracle's RK4).  The plain FP64 path is timed beside it
on the same batch.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Multi-GPU (torchrun): instances are independent, so every rank solves its
shard of one seeded global batch of 1024 x N instances (weak scaling, no
data-path collective); value = passing solves of all ranks / max time over
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SCP solves/s at defect<=1e-5 (batched FP32+refine; plain FP64 beside it); p50/p99 ms"
UNIT = "solves/s"
WORKLOAD = "mars_batch_1024_N100"
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM of Blackwell (compute capability 10.x)


def flops_per_node_iter(nx, nu, mirror_flops, refine=True):
    """FP32 arithmetic of one ADMM iteration at one node (FMA = 2 flops).

    Step 1: A^T w, B^T w (2 nx n), two triangular solves (2 n (n+1));
    refinement: H xi via A xi + B u, A^T v, B^T v (4 nx n) + 4 n, two more
    solves; propagation A x + B u + c (2 nx n); Steps 2-4: 12 flops per
    state component, 6 per control component, plus the mirror sets."""
    n = nx + nu
    f = 2 * nx * n + 2 * n * (n + 1) + 2 * nx * n + 12 * nx + 6 * nu + mirror_flops
    if refine:
        f += 4 * nx * n + 4 * n + 2 * n * (n + 1)
    return f


def flops_per_node_scp(nx, nu, f_flops):
    """Arithmetic of the once-per-SCP-iteration work at one node i < N (FMA = 2
    flops), counted by the dense formulas: the forward-mode linearisation
    through four RK4 stages (each stage f_x times the n_x x n tangent and f_u,
    the stage updates, then the four-term combination), the assembly of the
    symmetric H (the n(n+1)/2 entries of [A B]^T [A B], 2 n_x each), its
    Cholesky factor (n^3 / 3) and the cached inverse (2 n^3 / 3), and the RK4
    rollout of the candidate (four f evaluations, 2 n_x per stage update and
    combination term; double-float operations counted as one flop each).  For
    the 3-DOF Mars model this gives ~7.2 kflop, the ~8 kflop per node and SCP
    iteration (linearise + factor) of the scope table's measurement rules."""
    n = nx + nu
    lin = 4 * (2 * nx * nx * n + 2 * nx * nu + 2 * nx * n + f_flops) + 8 * nx * n
    assemble = n * (n + 1) // 2 * 2 * nx
    factor = n ** 3 // 3 + 2 * n ** 3 // 3
    rollout = 4 * (f_flops + 2 * nx) + 8 * nx
    return lin + assemble + factor + rollout


MARS7_F_FLOPS = 20   # one evaluation of the 3-DOF Mars dynamics: T/m (3 div + 3 add g), |T| and the mass rate


def mars_mirror_flops():
    # cone (|y|, compare, scale: ~30), ball (~20), half-space (~14) with their duals and RHS terms
    return 64


# what builds and launches the Mars FP32 fused kernel: its translation unit, the headers
# it includes and the host code that lays out and launches it
TRAFFIC_SOURCES = ("include/ucn.h",) + tuple("paper_2603_10711_gb300/csrc/" + f for f in (
    "ucn_api.cu", "ucn_df.cuh", "ucn_internal.h", "ucn_kernels.cuh", "ucn_lanes.cuh", "ucn_launch.cuh",
    "ucn_mars32.cu", "ucn_mars32_3.cu", "ucn_math.cuh", "ucn_pair.cuh"))


def kernel_sources_sha256():
    """Hash of TRAFFIC_SOURCES with their comments and blank lines removed, so
    that a change of documentation alone keeps the recorded traffic valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for p in TRAFFIC_SOURCES:
        text = open(os.path.join(ROOT, p), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(os.path.basename(p).encode())
        h.update(text.encode())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes of one batch solve (the fused kernel's launches of one
    ucn_scp_solve) from the committed ncu capture, or None when the kernel
    sources changed since that capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "scp_kernel_traffic.json")))
    except Exception:
        return None
    return rec["traffic_bytes_per_solve"] if rec.get("sources_sha256") == kernel_sources_sha256() else None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="ucn_clocks_gpu%d_" % gpu_index, suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        try:
            os.remove(self.path)
        except OSError:
            pass
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if len(r) > 5 + k and "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_over_ranks(total_time, passed, device):
    """Whole-job figures of a weak-scaling run: the slowest rank's time and the
    passed solves of all ranks (a control-path reduction; the solves share no data)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_time), float(passed)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def shard_bounds(batch, rank, world):
    """Contiguous instance range [lo, hi) of `rank` when one batch is split over ranks."""
    per, extra = divmod(batch, world)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def make_problem(args, rank=0, world=1):
    """The rank's share of one seeded global batch of args.batch x world
    instances (weak scaling: args.batch instances per rank; with one rank, the
    whole batch)."""
    over = {}
    if args.scp_iters:
        over = dict(scp_iters=args.scp_iters, stop=0)
    if getattr(args, "admm_iters", 0):
        over["admm_iters"] = args.admm_iters
    total = args.batch * world
    if getattr(args, "workload", "mars") == "quad_box":
        prob = W.quad_box(total, seed=2, settings=over)
    elif getattr(args, "workload", "mars") == "quad40":
        prob = W.quad_box(total, seed=2, N_range=(40, 40), obs_range=(8, 8), settings=over)
    else:
        prob = W.mars_batch(total, seed=1, settings=over)
    if world == 1:
        return prob
    lo, hi = shard_bounds(total, rank, world)
    return prob.subset(np.arange(lo, hi))


def run_kernel_only(args):
    """Only the FP32 fused kernel on the chosen batch (for profiler captures)."""
    import torch
    from paper_2603_10711_gb300 import ucn
    prob = make_problem(args)
    solver = ucn.Solver(prob, precision=ucn.UCN_PREC_FP64 if args.fp64 else ucn.UCN_PREC_FP32_REFINE)
    if args.lanes:
        ucn.ucn_problem_set_lanes(solver.handle, args.lanes)
    x0, u0 = solver.tensor(prob.xguess), solver.tensor(prob.uguess)
    for _ in range(args.warmup):
        solver.scp_solve(x0, u0)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(); solver.scp_solve(x0, u0); e1.record(); e1.synchronize()
        times.append(e0.elapsed_time(e1))
    st = solver.stats_host()
    solver.close()
    return {"mode": "kernel", "batch": prob.batch, "ms": times, "scp_iters_mean": float(st["scp_iters"].mean()),
            "pass_rate": float(np.mean(st["defect"] <= 1e-5))}


def run_ours(args, rank, world):
    import torch
    from paper_2603_10711_gb300 import ucn

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prob = make_problem(args, rank, world)
    B = prob.batch
    solver = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE, device=dev)
    stream = torch.cuda.current_stream(dev)
    x0 = solver.tensor(prob.xguess)
    u0 = solver.tensor(prob.uguess)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step():
        solver.scp_solve(x0, u0)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    times, passed, lat, nodeiters, nodescp = [], 0, [], 0, 0
    sampler = ClockSampler(dev.index)
    with sampler:
        for _ in range(args.steps):
            flush.fill_(1.0)                       # evict the batch from L2 between steps
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            st = solver.stats_host()
            passed += int(np.sum(st["defect"] <= 1e-5))
            t0 = st["t_start_ns"].min()
            lat.extend(((st["t_end_ns"] - t0) / 1e6).tolist())
            nodeiters += int(np.sum(st["scp_iters"].astype(np.int64) * (prob.N.astype(np.int64) + 1))) * int(prob.settings["admm_iters"])
            nodescp += int(np.sum(st["scp_iters"].astype(np.int64) * prob.N.astype(np.int64)))
    torch.cuda.synchronize()
    # the last timed step's results, for the parity check against the oracle
    x_last, u_last, st_timed = solver.x_out.cpu().numpy(), solver.u_out.cpu().numpy(), solver.stats_host()
    total = sum(times)
    if world > 1:
        total, passed_all = reduce_over_ranks(total, passed, dev)
    else:
        passed_all = passed
    value = passed_all / total
    clocks = sampler.summary()

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    xh = torch.from_numpy(np.ascontiguousarray(prob.xguess)).pin_memory()
    uh = torch.from_numpy(np.ascontiguousarray(prob.uguess)).pin_memory()
    xo_h = torch.empty(solver.x_out.shape, dtype=torch.float64).pin_memory()
    uo_h = torch.empty(solver.u_out.shape, dtype=torch.float64).pin_memory()
    so_h = torch.empty(solver.stats.shape, dtype=torch.uint8).pin_memory()
    e2e_times, e2e_pass = [], 0
    for _ in range(max(2, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x0.copy_(xh, non_blocking=True); u0.copy_(uh, non_blocking=True)
        solver.scp_solve(x0, u0)
        xo_h.copy_(solver.x_out, non_blocking=True); uo_h.copy_(solver.u_out, non_blocking=True)
        so_h.copy_(solver.stats, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        e2e_times.append(time.perf_counter() - t0)
        st = np.frombuffer(so_h.numpy().tobytes(), dtype=ucn.STATS_DTYPE)
        e2e_pass += int(np.sum(st["defect"] <= 1e-5))
    h2d = xh.numel() * 8 + uh.numel() * 8
    d2h = xo_h.numel() * 8 + uo_h.numel() * 8 + so_h.numel()

    # ---- plain FP64 path on the same batch (a few steps; it is the slow comparison path)
    s64 = ucn.Solver(prob, precision=ucn.UCN_PREC_FP64, device=dev)
    s64.scp_solve(x0, u0); torch.cuda.synchronize()
    t64, p64 = [], 0
    for _ in range(args.fp64_steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream); s64.scp_solve(x0, u0); e1.record(stream); e1.synchronize()
        t64.append(e0.elapsed_time(e1) / 1e3)
        p64 += int(np.sum(s64.stats_host()["defect"] <= 1e-5))
    st64 = s64.stats_host()
    s64.close()

    serving_out = run_serving(args) if (args.serving_requests > 0 and world == 1) else None
    batching_out = run_batching(args) if (args.batching_batch > 0 and world == 1) else None
    rho_out = run_rho_study(args) if (args.rho_study_batch > 0 and world == 1) else None
    scenario_out = run_scenarios(args) if (args.scenario_steps > 0 and world == 1) else None
    single_out = run_single_quad(args) if (args.single_solves > 0 and world == 1) else None

    flops_ni = flops_per_node_iter(prob.nx, prob.nu, mars_mirror_flops())
    flops_ns = flops_per_node_scp(prob.nx, prob.nu, MARS7_F_FLOPS)
    flops_admm = nodeiters / args.steps * flops_ni
    flops_launch = flops_admm + nodescp / args.steps * flops_ns
    avg = total / args.steps if world == 1 else sum(times) / len(times)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tf = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops_launch / avg / 1e12
    st_last = solver.stats_host()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (ADMM) + f32-pair double-float (nominal, rollout, defects, merits) + f64 (acceptance test, results)",
        "data": "synthetic (seeded Mars descent dispersions)",
        "config": {"workload": WORKLOAD, "instances_per_gpu": B, "horizon": 100, "nx": 7, "nu": 3,
                   "admm_iters_per_scp": int(prob.settings["admm_iters"]), "scp_iter_cap": int(prob.settings["scp_iters"]),
                   "rho": "%g -> %g geometric" % (prob.settings["rho_geo"], prob.settings["rho_final"]),
                   "stop": "defect <= 1e-5", "l2": "flushed (256 MB write) before each step",
                   "parallelism": "one CTA per instance, one thread per node; ranks hold independent batches"},
        "pass_rate": passed / (B * args.steps),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "definition": "per solve: instance end - first instance start within its launch"},
        "scp_iters_mean": float(st_last["scp_iters"].mean()),
        "fp64_plain": {"value": p64 / sum(t64), "unit": UNIT, "ms_per_step": 1e3 * sum(t64) / len(t64),
                       "pass_rate": p64 / (B * len(t64)), "scp_iters_mean": float(st64["scp_iters"].mean())},
        "e2e": {"value": e2e_pass / sum(e2e_times), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf, "traffic": recorded_traffic(),
                     "traffic_unit": "bytes per batch solve: the fused kernel's launches of one ucn_scp_solve "
                                     "(ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                     "peak_note": "derived: %d SMs (read from the device) x %d FP32 lanes x 2 x %.0f MHz (max SM clock, "
                                  "MEASURED_PEAKS.json)" % (sm_count, FP32_LANES_PER_SM, sm_max),
                     "algorithmic_flops_per_node_iter": flops_ni, "node_iters_per_launch": nodeiters / args.steps,
                     "algorithmic_flops_per_node_scp_iter": flops_ns, "node_scp_iters_per_launch": nodescp / args.steps,
                     "achieved_admm_only": flops_admm / avg / 1e12,
                     "definition": "achieved = (flops per node and ADMM iteration x node-iterations + flops per node "
                                   "i < N and SCP iteration x node-SCP-iterations) of one batch solve / its CUDA-event "
                                   "time; achieved_admm_only counts the ADMM iterations alone"},
        "gpu_launches": args.steps * ucn.ucn_problem_last_launches(solver.handle),
        "clocks": clocks,
    }
    if single_out is not None:
        out["single_quad"] = single_out
    if serving_out is not None:
        out["serving"] = serving_out
    if scenario_out is not None:
        out["scenario_mpc"] = scenario_out
    if batching_out is not None:
        out["batching"] = batching_out
    if rho_out is not None:
        out["rho_study"] = rho_out
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"], out["parity"] = cpu_baseline(args, (x_last, u_last, st_timed))
    solver.close()
    return out


def run_serving(args):
    """Continuous batching of a mixed Poisson request stream (70% quadrotor,
    30% Mars descent) in FP32 at each arrival rate of --serving-rates (the
    configuration's 2k-20k req/s), by pump launches and by the device-resident
    request loop, and the stream's head solved one request at a time in FP64
    (the plain per-request path).  Capacity = the largest
    completed-solve rate; knee = the first rate at which the completed rate
    falls below 90% of the arrival rate (the server saturates)."""
    from paper_2603_10711_gb300 import serving, ucn
    qs = W.quad_box(1).settings
    # Mars requests run up to N = 200: the batch's 60 x 40 schedule converges up to N = 150,
    # longer horizons need more ADMM iterations per SCP iteration (80 x 60 passes up to 200)
    ms = dict(W.mars_batch(1).settings, rho_final=1e7, scp_iters=80, admm_iters=60)

    # one server per model and horizon bucket: a server's CTA size and node layout follow
    # its longest horizon, so short requests run in small CTAs with their records in
    # shared memory (a quadrotor node with 30 obstacle mirrors takes ~3 KB: up to 72
    # nodes fit one CTA's shared memory)
    buckets = {1: (40, 72, 120), 2: (100, 200)}
    route = serving.horizon_route(buckets)

    def servers(prec, slots):
        sv = {}
        for h in buckets[1]:
            sv[(1, h)] = serving.Server(1, prec, max_slots=slots, max_horizon=h, max_obs=30, lanes=8, settings=qs)
        for h in buckets[2]:
            sv[(2, h)] = serving.Server(2, prec, max_slots=slots, max_horizon=h, lanes=8, settings=ms)
        return sv

    rates = [float(r) for r in args.serving_rates.split(",")]
    sv = servers(ucn.UCN_PREC_FP32_REFINE, 512)
    serving.run_stream(W.serving_stream(32, rate=rates[0], seed=4), sv, route=route)    # warm-up
    # one set of requests; the arrival gaps are Exp(rate) = Exp(1) / rate of the same draws
    base = W.serving_stream(args.serving_requests, rate=1.0, seed=4)
    sweep = []
    for rate in rates:
        stream = [(t / rate, p) for t, p in base]
        r = serving.run_stream(stream, sv, route=route)
        sweep.append(dict(r, arrival_rate_per_s=rate, requests=len(stream)))
    for s in sv.values():
        s.close()
    knee = next((r["arrival_rate_per_s"] for r in sweep if r["solves_per_s"] < 0.9 * r["arrival_rate_per_s"]), None)

    # the same streams through the device-resident request loop: one persistent kernel
    # per server whose CTAs claim each request as it is submitted (no pump launches).
    # The loops run at the same time, so each holds a share of the device: server i
    # needs c_i = rate_i x t_i CTAs to keep up (t_i: its mean device time per solve,
    # measured in the pump sweep's first stream) and c_i / cap_i of the device (cap_i:
    # its CTAs that fit at once), so c_i = cap_i x s_i with s_i proportional to
    # n_i t_i / cap_i, 90% of the device in all
    sv = servers(ucn.UCN_PREC_FP32_REFINE, 512)
    busy = sweep[0]["solve_ms_by_server"]
    caps = {k: srv.loop_capacity() for k, srv in sv.items()}
    name = serving.server_name
    need = {k: (busy[name(k)][0] * busy[name(k)][1] / caps[k] if name(k) in busy else 0.0) for k in sv}
    total = sum(need.values())
    loop_ctas = {}
    for k, srv in sv.items():
        loop_ctas[k] = max(1, int(0.9 * caps[k] * need[k] / total))
        srv.loop_start(ctas=loop_ctas[k], idle_s=2.0)
    serving.run_stream(W.serving_stream(32, rate=rates[0], seed=4), sv, route=route)    # warm-up
    loop_sweep = []
    for rate in rates:
        stream = [(t / rate, p) for t, p in base]
        r = serving.run_stream(stream, sv, route=route)
        loop_sweep.append(dict(r, arrival_rate_per_s=rate, requests=len(stream)))
    loop_launches = 0
    for s in sv.values():
        s.loop_stop()
        loop_launches += s.loop_launches()
        s.close()
    loop_knee = next((r["arrival_rate_per_s"] for r in loop_sweep if r["solves_per_s"] < 0.9 * r["arrival_rate_per_s"]),
                     None)
    stream = base
    sv = servers(ucn.UCN_PREC_FP64, 4)
    n64 = min(len(stream), args.serving_fp64_requests)
    fp64 = serving.run_stream([(0.0, p) for _, p in stream[:n64]], sv, max_inflight=1, route=route)
    for s in sv.values():
        s.close()
    return {"mix": "70% quad N 30-120, 5-30 obstacles / 30% Mars N 50-200",
            "servers": "one per model and horizon bucket: quadrotor N <= 40 / 72 / 120, Mars N <= 100 / 200",
            "fp32_continuous": sweep,
            "capacity_solves_per_s": max(r["solves_per_s"] for r in sweep), "knee_arrival_rate_per_s": knee,
            "fp32_device_loop": loop_sweep,
            "device_loop_capacity_solves_per_s": max(r["solves_per_s"] for r in loop_sweep),
            "device_loop_knee_arrival_rate_per_s": loop_knee,
            "device_loop_ctas": {name(k): [v, caps[k]] for k, v in loop_ctas.items()},
            "device_loop_launches": loop_launches,
            "fp64_per_request": dict(fp64, requests=n64),
            "latency": "arrival -> result collected (host clock)"}


def run_single_quad(args):
    """The single quadrotor (12 states, N = 50, 5 obstacles, goal drawn with seed
    0) in the plain FP64 path with the fixed 15 SCP x 200 ADMM schedule, one
    instance per launch, timed per solve (CUDA events, after warm-up); the FP32
    path with refinement on the same problem beside it."""
    import torch
    from paper_2603_10711_gb300 import ucn
    prob = W.quad_path(1, seed=0)
    out = {"workload": "quad_path_1_N50_obs5", "scp_iters": int(prob.settings["scp_iters"]),
           "admm_iters": int(prob.settings["admm_iters"]), "solves": args.single_solves}
    for name, prec in (("fp64_plain", ucn.UCN_PREC_FP64), ("fp32_refine", ucn.UCN_PREC_FP32_REFINE)):
        s = ucn.Solver(prob, precision=prec)
        x0, u0 = s.tensor(prob.xguess), s.tensor(prob.uguess)
        for _ in range(3):
            s.scp_solve(x0, u0)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.single_solves):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(); s.scp_solve(x0, u0); e1.record(); e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = s.stats_host()
        s.close()
        out[name] = {"ms_p50": float(np.percentile(ms, 50)), "ms_p99": float(np.percentile(ms, 99)),
                     "solves_per_s": 1e3 / float(np.mean(ms)), "defect": float(st["defect"][0]),
                     "status": int(st["status"][0])}
    return out


def run_batching(args):
    """Uneven-horizon batching: 4096 quadrotors, N ~ U{40..120}, 10-30 obstacles,
    FP32 + refinement.  The autotuner picks the size-class split and threads per
    node on a 608-instance sample; the batch is then solved as one plain launch
    (library defaults) and as the tuned classes replayed from a CUDA graph."""
    import torch
    from paper_2603_10711_gb300 import batching, ucn
    prob = W.quad_box(args.batching_batch, seed=2)
    t0 = time.perf_counter()
    cfg, timings = batching.autotune(prob, cache_path=None)
    tune_s = time.perf_counter() - t0
    out = {"workload": "quad_box_%d_N40-120_obs10-30" % prob.batch, "autotuned": cfg, "autotune_s": tune_s,
           "candidates_ms": {k: 1e3 * v for k, v in timings.items()}}
    for name, kw in (("default_single_launch", dict(splits=[])), ("tuned_graph", dict(splits=cfg["splits"], lanes=cfg["lanes"]))):
        cs = batching.ClassedSolver(prob, **kw)
        if name == "tuned_graph":
            cs.capture()
        cs.solve(); torch.cuda.synchronize()
        ms = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(); cs.solve(); e1.record(); e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = cs.stats()
        passed = int(np.sum(st["defect"] <= 1e-5))
        out[name] = {"ms": min(ms), "solves_per_s": passed / (min(ms) / 1e3), "pass_rate": passed / prob.batch,
                     "scp_iters_mean": float(st["scp_iters"].mean())}
        cs.close()
    # the plain FP64 path on the same batch, one launch (library defaults)
    s64 = ucn.Solver(prob, precision=ucn.UCN_PREC_FP64)
    x0, u0 = s64.tensor(prob.xguess), s64.tensor(prob.uguess)
    s64.scp_solve(x0, u0); torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(); s64.scp_solve(x0, u0); e1.record(); e1.synchronize()
    ms64 = e0.elapsed_time(e1)
    st = s64.stats_host()
    s64.close()
    passed = int(np.sum(st["defect"] <= 1e-5))
    out["fp64_plain_single_launch"] = {"ms": ms64, "solves_per_s": passed / (ms64 / 1e3), "pass_rate": passed / prob.batch,
                                       "scp_iters_mean": float(st["scp_iters"].mean())}
    return out


def run_rho_study(args):
    """The paper's penalty-schedule study (Sec. IV-A2) on the 13-state quaternion
    quadrotor: all three penalties from 1 to rho_f geometrically over 20 SCP
    iterations, rho_f in {1e3, 1e4, 1e5, 1e6}, 100 or 250 ADMM iterations per
    SCP iteration; a batch of study tasks (obstacle placements drawn per
    instance) solved in FP32 + refinement.  Reports the final defect and cost."""
    import torch
    from paper_2603_10711_gb300 import ucn
    rows = []
    for admm in (100, 250):
        for rf in (1e3, 1e4, 1e5, 1e6):
            prob = W.quat_study(args.rho_study_batch, seed=5, rho_final=rf, admm_iters=admm)
            s = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE)
            x0, u0 = s.tensor(prob.xguess), s.tensor(prob.uguess)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(); s.scp_solve(x0, u0); e1.record(); e1.synchronize()
            st = s.stats_host()
            s.close()
            rows.append({"rho_final": rf, "admm_iters": admm, "defect_median": float(np.median(st["defect"])),
                         "defect_max": float(st["defect"].max()), "cost_mean": float(st["cost"].mean()),
                         "ms": e0.elapsed_time(e1)})
    return {"workload": "quat_study_%d_N50" % args.rho_study_batch, "scp_iters": 20, "rho0": 1.0, "rows": rows}


def run_scenarios(args):
    """Scenario-based robust MPC (Sec. IV-A): P quadrotor problems x K scenarios
    (mass, drag) sharing the first control, N = 40, 8 obstacles; a receding
    horizon of S steps, each one grouped solve (thread-block clusters, FP32 +
    refinement) and one shift that applies the shared control and warm-starts
    the next solve.  The plain FP64 path runs the first (cold) step of the
    first `--scenario-fp64-problems` problems."""
    import torch
    from paper_2603_10711_gb300 import ucn
    P, K, S = args.scenario_problems, args.scenario_count, args.scenario_steps
    prob = W.scenario_mpc(P, K, seed=3, N=40, n_obs=8)
    for prec in (ucn.UCN_PREC_FP32_REFINE, ucn.UCN_PREC_FP64):     # warm-up: module load, cluster set-up
        w = ucn.Solver(W.scenario_mpc(2, K, seed=13, N=40, n_obs=8, settings=dict(scp_iters=2, admm_iters=20)),
                       precision=prec)
        w.scp_solve(); torch.cuda.synchronize(); w.close()
    kc = K if K <= 16 else (2 if K % 2 == 0 else 1)     # the library's cluster size for a group of K
    goal = prob.xtarget[::K, :3]
    d0 = np.linalg.norm(prob.xinit[::K, :3] - goal, axis=1)
    s = ucn.Solver(prob, precision=ucn.UCN_PREC_FP32_REFINE)
    x0, u0 = s.tensor(prob.xguess), s.tensor(prob.uguess)
    xg, ug = x0, u0
    stream = torch.cuda.current_stream()
    step_ms, passed, iters = [], 0, []
    for k in range(S):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.scp_solve(xg, ug)
        xg, ug = s.mpc_shift()
        e1.record(stream); e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = s.stats_host()
        passed += int(np.sum(st["defect"] <= 1e-5))
        iters.append(float(st["scp_iters"].mean()))
    d1 = np.linalg.norm(xg.cpu().numpy()[prob.xoff[::K], :3] - goal, axis=1)
    s.close()
    total = sum(step_ms) / 1e3
    # plain FP64: the cold first step of the first P64 problems
    P64 = min(P, args.scenario_fp64_problems)
    p64 = W.scenario_mpc(P, K, seed=3, N=40, n_obs=8).subset(np.arange(P64 * K))
    s64 = ucn.Solver(p64, precision=ucn.UCN_PREC_FP64)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream); s64.scp_solve(); e1.record(stream); e1.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    st64 = s64.stats_host()
    s64.close()
    return {"workload": "scenario_mpc_%dx%d_N40" % (P, K), "problems": P, "scenarios": K, "mpc_steps": S,
            "groups": "%d CTAs per group: %d thread-block cluster(s) of %d" % (K, K // kc, kc),
            "problem_steps_per_s": P * S / total, "scenario_solves_per_s": P * K * S / total,
            "step_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                        "first_cold": step_ms[0]},
            "pass_rate": passed / (P * K * S), "scp_iters_mean_per_step": iters,
            "goal_distance_m": {"start_mean": float(d0.mean()), "end_mean": float(d1.mean())},
            "fp64_plain_cold_step": {"problems": P64, "ms": 1e3 * t64, "scenario_solves_per_s": P64 * K / t64,
                                     "pass_rate": float(np.mean(st64["defect"] <= 1e-5)),
                                     "scp_iters_mean": float(st64["scp_iters"].mean())},
            "fp32_cold_step_ms": step_ms[0]}


def oracle_sample(args, n=None):
    """The FP64 CPU oracle on a bounded sample of the same workload (n instances,
    evenly spaced; default --cpu-sample).  Returns (passed, n, seconds, threads,
    sample indices, the oracle's (x, u, stats), the sample problem)."""
    import oracle
    prob = W.mars_batch(args.batch, seed=1)
    threads = oracle.max_threads()
    n = min(args.batch, max(threads, args.cpu_sample if n is None else n))
    idx = np.arange(n) * (prob.batch // n)
    sub = prob.subset(idx)
    t0 = time.perf_counter()
    xr, ur, st, _ = oracle.scp_solve(sub, nthreads=threads)
    dt = time.perf_counter() - t0
    passed = int(np.sum(st[:, 0] <= 1e-5))
    return passed, n, dt, threads, idx, (xr, ur, st), sub


def cpu_baseline(args, gpu_result=None):
    """The oracle timed on the host cores, and -- on the same instances, from its
    trajectories -- the parity of the GPU's last timed step: every sampled
    trajectory against the oracle's at 1e-4 after the same SCP iteration count,
    and the FP64 defect of the GPU's returned doubles by the oracle's RK4."""
    passed, n, dt, threads, idx, ref, sub = oracle_sample(args)
    base = {"value": passed / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of the %d Mars instances (every %d-th), %.1f s, %d passed" % (n, args.batch, args.batch // n, dt, passed)}
    import oracle
    # the same oracle on one host core, on the first 16 instances of that sample
    one = sub.subset(np.arange(min(16, n)))
    t0 = time.perf_counter()
    st1 = oracle.scp_solve(one, nthreads=1)[2]
    dt1 = time.perf_counter() - t0
    base["single_core"] = {"value": float(np.sum(st1[:, 0] <= 1e-5)) / dt1, "unit": UNIT, "cores": 1,
                           "sample": "the first %d instances of the sample, %.2f s" % (one.batch, dt1)}
    if gpu_result is None:
        return base, None
    xg, ug, st = gpu_result
    prob = W.mars_batch(args.batch, seed=1)
    xs = np.concatenate([xg[prob.xoff[b]:prob.xoff[b] + prob.N[b] + 1] for b in idx])
    us = np.concatenate([ug[prob.uoff[b]:prob.uoff[b] + prob.N[b]] for b in idx])
    t0 = time.perf_counter()
    r = oracle.compare_batch(sub, xs, us, st["scp_iters"][idx], ref, 1e-4, nthreads=threads)
    same = np.ones(n, dtype=bool)
    same[r["mismatch"]] = False
    parity = dict(r["summary"])
    def spread(v):
        # per-instance values: percentiles and a histogram by decade (upper edges)
        v = np.asarray(v, dtype=np.float64)
        edges = [1e-12, 1e-11, 1e-10, 1e-9, 1e-8, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, np.inf]
        counts = np.histogram(v, bins=[0.0] + edges)[0]
        return {"p50": float(np.percentile(v, 50)), "p90": float(np.percentile(v, 90)),
                "p99": float(np.percentile(v, 99)), "max": float(v.max()),
                "count_below": {("%.0e" % e if np.isfinite(e) else "inf"): int(c) for e, c in zip(edges, counts)}}
    parity.update({
        "per_instance_rel_err": spread(r["err"]),
        "per_instance_fp64_defect": spread(r["fp64_defect"]),
        "max_rel_err_same_iters_as_oracle": float(r["err"][same].max()) if same.any() else None,
        "gpu_defect_vs_oracle_rk4_max_abs": float(np.abs(st["defect"][idx] - r["fp64_defect"]).max()),
        "check_s": time.perf_counter() - t0,
        "definition": "per instance |gpu - oracle|_max / max(1, |oracle|_max) over x and u of the returned "
                      "trajectory, the oracle (FP64 CPU) solving the same inputs; where the stop test "
                      "(defect <= 1e-5) ended the two solves after different SCP iteration counts the "
                      "oracle is re-run to the GPU's count (scp_iters_mismatch); fp64_defect_* = max_i "
                      "|RK4(x_i, u_i) - x_{i+1}|_inf of the GPU's returned doubles by the oracle's FP64 RK4"})
    return base, parity


def run_reference(args, rank, world):
    if rank != 0:
        return None
    times, passed_all, n_all = [], 0, 0
    for _ in range(args.warmup):
        pass   # the oracle has no warm state; warm-up steps are not needed on the CPU
    for _ in range(args.steps):
        passed, n, dt, threads = oracle_sample(args, args.ref_sample)[:4]
        times.append(dt); passed_all += passed; n_all += n
    value = passed_all / sum(times)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Mars descent dispersions)",
            "config": {"workload": WORKLOAD, "instances_per_step": n_all // args.steps},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d Mars instances per step on %d host threads" % (n_all // args.steps, threads)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "pass_rate": passed_all / max(1, n_all)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample", type=int, default=1024)
    ap.add_argument("--ref-sample", type=int, default=128, help="instances per step of the reference (oracle) arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=8000,
                    help="requests of each serving stream (0: skip); long enough that the drain after the last "
                         "arrival weighs little in the completed rate")
    ap.add_argument("--serving-rates", default="2000,5000,10000,20000", help="Poisson arrival rates of the serving sweep")
    ap.add_argument("--serving-fp64-requests", type=int, default=16)
    ap.add_argument("--batching-batch", type=int, default=4096, help="uneven quadrotor batch (0: skip the section)")
    ap.add_argument("--rho-study-batch", type=int, default=256, help="quaternion study tasks per setting (0: skip)")
    ap.add_argument("--scenario-problems", type=int, default=256)
    ap.add_argument("--scenario-count", type=int, default=64, help="scenarios per problem (group size)")
    ap.add_argument("--scenario-steps", type=int, default=50, help="receding-horizon steps (0: skip the section)")
    ap.add_argument("--single-solves", type=int, default=20, help="timed solves of the single quadrotor (0: skip)")
    ap.add_argument("--scenario-fp64-problems", type=int, default=64)
    ap.add_argument("--mode", default="full", choices=["full", "kernel", "scenario", "batching", "rho_study", "serving", "single"],
                    help="kernel: time only the fused kernel (profiler captures)")
    ap.add_argument("--scp-iters", type=int, default=0, help="fixed SCP iteration count (0: the workload's cap + stop test)")
    ap.add_argument("--admm-iters", type=int, default=0, help="kernel mode: ADMM iterations per SCP iteration (0: the workload's)")
    ap.add_argument("--fp64", action="store_true", help="kernel mode: the FP64 plain path")
    ap.add_argument("--workload", default="mars", choices=["mars", "quad_box", "quad40"],
                    help="kernel mode: mars (1024-instance Mars batch), quad_box (uneven quadrotor batch) "
                         "or quad40 (quadrotors with N = 40 and 8 obstacles)")
    ap.add_argument("--lanes", type=int, default=0, help="kernel mode: threads per node (0: the library default)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.mode == "kernel":
        out = run_kernel_only(args)
    elif args.mode == "scenario":
        out = run_scenarios(args)
    elif args.mode == "batching":
        out = run_batching(args)
    elif args.mode == "rho_study":
        out = run_rho_study(args)
    elif args.mode == "serving":
        out = run_serving(args)
    elif args.mode == "single":
        out = run_single_quad(args)
    elif args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
