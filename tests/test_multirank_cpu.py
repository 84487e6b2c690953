"""The multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1.
Each rank owns a contiguous, disjoint slice of the trajectory index space (weak
scaling, no data-path collective) and the step time reported is the maximum
over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2301_03989_gb300 import workloads as W
    n_per = 6
    wall = W.config2(M=n_per * world)
    lo, hi = bench.shard(wall.n_ic, world, rank)
    w = wall.subset(np.arange(lo, hi))
    t_max = bench.max_over_ranks(10.0 + rank, world)
    out.put((rank, lo, hi, w.x0.copy(), t_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_max():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in range(world)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2301_03989_gb300 import workloads as W
    full = W.config2(M=12).x0
    assert [(r[1], r[2]) for r in res] == [(0, 6), (6, 12)]          # disjoint, covering
    np.testing.assert_array_equal(np.concatenate([r[3] for r in res]), full)
    assert all(r[4] == 11.0 for r in res)                            # max over ranks
