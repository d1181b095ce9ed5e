"""Multi-rank path of the benchmark on CPU: two gloo ranks, each with its own replica,
whole-job throughput = all ranks' pairs over the slowest rank (no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.config_hull_vs_primitive(n=6, seed=bench.rank_seed(rank))
        local_ms = 10.0 + 5.0 * rank

        def max_over_ranks(v):
            t = torch.tensor([v], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        value, ms = bench.aggregate(local_ms, w.n_pairs, 3, world, max_over_ranks)
        q.put((rank, value, ms, w.poses[0].tolist(), w.n_pairs))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, v0, ms0, pose0, n0), (_, v1, ms1, pose1, n1) = res
    assert ms0 == ms1 == 15.0                      # the slowest rank sets the time
    assert v0 == v1 == pytest.approx(2 * n0 * 3 / 15e-3)
    assert n0 == n1 and not np.allclose(pose0, pose1)   # independent replicas of equal size
