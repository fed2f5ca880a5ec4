"""Scheduling of uneven-horizon batches: size classes, autotuning, CUDA graphs.

A batch whose horizons differ (e.g. N in [40, 120]) is split into size
classes by horizon.  Each class is its own ucn_problem, so its CTA size
(nodes per block, one thread per node) and its node-record layout follow its
own longest horizon: short quadrotor instances then fit in shared memory and
run fully on chip, long ones use the global-memory workspace.  The classes'
fused solves are launched on separate streams and overlap on the device; the
whole multi-stream solve can be captured once in a CUDA graph and replayed.

The split points are picked by `autotune`, which times each candidate
split on a sample of the batch and caches the winner per problem signature.
Within a class the fused kernel takes instances largest-first (see
``ucn_problem_set_order``).

Everything here is host-side orchestration of the C ABI: every step of the
method runs in the CUDA library.
"""
from __future__ import annotations

import json
import os
import time
from typing import List, Optional, Sequence

import numpy as np

from . import ucn

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ucn_autotune_v2.json")


def class_indices(N: np.ndarray, splits: Sequence[int]) -> List[np.ndarray]:
    """Instance indices of each size class: class k holds N+1 in (s_{k-1}, s_k]."""
    bounds = [0] + sorted(int(s) for s in splits) + [1 << 30]
    out = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        idx = np.nonzero((N + 1 > lo) & (N + 1 <= hi))[0]
        if idx.size:
            out.append(idx)
    return out


class ClassedSolver:
    """The fused SCP solve of one batch, split into size classes."""

    def __init__(self, prob, splits: Sequence[int] = (), precision=ucn.UCN_PREC_FP32_REFINE, device="cuda",
                 lanes: int = 0):
        import torch
        self.prob = prob
        self.splits = list(splits)
        self.device = torch.device(device)
        self.classes = class_indices(np.asarray(prob.N), self.splits)
        self.subs = [prob.subset(idx) for idx in self.classes]
        self.solvers = [ucn.Solver(sp, precision=precision, device=device) for sp in self.subs]
        if lanes:
            # threads per node where the class allows it (4 needs a quadrotor class of <= 128 nodes)
            for s in self.solvers:
                try:
                    ucn.ucn_problem_set_lanes(s.handle, lanes)
                except ucn.UcnError:
                    ucn.ucn_problem_set_lanes(s.handle, 1)
        self.x0 = [s.tensor(sp.xguess) for s, sp in zip(self.solvers, self.subs)]
        self.u0 = [s.tensor(sp.uguess) for s, sp in zip(self.solvers, self.subs)]
        self.streams = [torch.cuda.Stream(device=self.device) for _ in self.solvers]
        self.graph = None

    def close(self):
        for s in self.solvers:
            s.close()

    def launch(self):
        """Enqueue every class on its own stream, joined back to the current stream."""
        import torch
        cur = torch.cuda.current_stream(self.device)
        start = torch.cuda.Event()
        start.record(cur)
        ends = []
        for s, st, x0, u0 in zip(self.solvers, self.streams, self.x0, self.u0):
            st.wait_event(start)
            with torch.cuda.stream(st):
                s.scp_solve(x0, u0, stream=st)
            e = torch.cuda.Event()
            e.record(st)
            ends.append(e)
        for e in ends:
            cur.wait_event(e)

    def capture(self):
        """Capture the multi-stream solve in a CUDA graph (call once, then `replay`)."""
        import torch
        self.launch()                      # first launches happen outside capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch()
        self.graph = g
        return g

    def solve(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.launch()

    def stats(self) -> np.ndarray:
        """Per-instance stats in the batch's instance order."""
        out = np.zeros(self.prob.batch, dtype=ucn.STATS_DTYPE)
        for idx, s in zip(self.classes, self.solvers):
            out[idx] = s.stats_host()
        return out

    def trajectories(self):
        """(x, u) on the host, packed in the batch's order."""
        x = np.zeros((self.prob.total_x, self.prob.nx))
        u = np.zeros((self.prob.total_u, self.prob.nu))
        xo, uo, N = self.prob.xoff, self.prob.uoff, self.prob.N
        for idx, sp, s in zip(self.classes, self.subs, self.solvers):
            xs, us = s.x_out.cpu().numpy(), s.u_out.cpu().numpy()
            for k, b in enumerate(idx):
                x[xo[b]:xo[b] + N[b] + 1] = xs[sp.xoff[k]:sp.xoff[k] + N[b] + 1]
                u[uo[b]:uo[b] + N[b]] = us[sp.uoff[k]:sp.uoff[k] + N[b]]
        return x, u


def signature(prob, precision) -> str:
    N = np.asarray(prob.N)
    return "m%d_p%d_B%d_N%d-%d_o%d" % (prob.model, precision, prob.batch, N.min(), N.max(), prob.max_obs)


def candidate_splits(prob) -> List[List[int]]:
    """No split, and one split at each multiple of 32 nodes inside the horizon range."""
    N = np.asarray(prob.N)
    lo, hi = int(N.min()) + 1, int(N.max()) + 1
    cands = [[]]
    for s in range(32, hi, 32):
        if lo <= s < hi:
            cands.append([s])
    return cands


def candidate_configs(prob) -> List[dict]:
    """Every split, with one and with four threads per node (quadrotor) -- the
    per-node parallelism the CTA size follows."""
    lanes = (1, 4) if int(prob.model) == ucn.UCN_MODEL_QUAD12 else (1,)
    return [{"splits": sp, "lanes": ln} for sp in candidate_splits(prob) for ln in lanes]


def autotune(prob, precision=ucn.UCN_PREC_FP32_REFINE, sample: int = 608, scp_iters: int = 3,
             cache_path: Optional[str] = DEFAULT_CACHE, device="cuda", verbose=False):
    """Pick the size-class split and threads per node with the shortest solve
    of a sample of the batch.

    Each candidate of `candidate_configs` runs `scp_iters` fixed SCP iterations
    (the iteration count only scales the time) on `sample` evenly spaced
    instances; the fastest is cached under the batch's signature.  Returns
    (config, timings), config = {"splits": [...], "lanes": n}."""
    import torch
    sig = signature(prob, precision)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if sig in cache:
        return cache[sig]["config"], cache[sig]["timings"]
    n = min(sample, prob.batch)
    sub = prob.subset(np.linspace(0, prob.batch - 1, n).astype(np.int64))
    sub.settings.update(dict(scp_iters=scp_iters, stop=0))
    timings = {}
    for cand in candidate_configs(sub):
        cs = ClassedSolver(sub, cand["splits"], precision=precision, device=device, lanes=cand["lanes"])
        cs.launch()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        cs.launch()
        torch.cuda.synchronize(device)
        timings[json.dumps(cand)] = time.perf_counter() - t0
        cs.close()
        if verbose:
            print("config", cand, "%.2f ms" % (1e3 * timings[json.dumps(cand)]))
    best = json.loads(min(timings, key=timings.get))
    if cache_path:
        cache[sig] = {"config": best, "timings": timings}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return best, timings
