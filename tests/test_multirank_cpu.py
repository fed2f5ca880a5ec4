"""The multi-rank path on CPU (gloo, world_size 2): every rank builds its
shard of one seeded global batch, and the benchmark's cross-rank reduction
combines the timing (max) and the solve counts (sum)."""
import argparse
import os
import socket

import numpy as np

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import workloads as W  # noqa: E402

ARGS = argparse.Namespace(batch=6, scp_iters=0, admm_iters=0, workload="mars")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shard = bench.make_problem(ARGS, rank, world)
        total, count = bench.reduce_over_ranks(1.5 + rank, shard.batch, torch.device("cpu"))
        q.put((rank, total, count, shard.xinit.tolist()))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, count, _ in out:
        assert total == 2.5                          # slowest rank
        assert count == 2 * ARGS.batch               # all ranks' instances
    # the two shards are the global batch, in order, without overlap
    whole = W.mars_batch(2 * ARGS.batch, seed=1)
    np.testing.assert_array_equal(np.concatenate([np.array(o[3]) for o in out]), whole.xinit)


@pytest.mark.parametrize("batch,world", [(1024, 2), (1024, 3), (5, 8), (7, 1)])
def test_shard_bounds_cover_the_batch(batch, world):
    seen = []
    for r in range(world):
        lo, hi = bench.shard_bounds(batch, r, world)
        assert 0 <= lo <= hi <= batch
        seen.extend(range(lo, hi))
    assert seen == list(range(batch))
