"""The benchmark's multi-GPU path is N independent replicas (no data-path collective): every rank runs its
own chains, the timed region's length is the maximum over ranks, and the job's rate is world x per-rank
units over that maximum.  Checked here with two gloo processes on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" (r + 1) seconds: every rank sees the slowest one
        t = bench.max_over_ranks(float(rank + 1), world, device="cpu")
        out[rank] = (t, bench.replicas_rate(world, 5, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][0] == 2.0
        assert res[r][1] == pytest.approx(5.0)   # 2 replicas x 5 steps in 2 s


def test_replicas_run_their_own_chains():
    import bench
    from paper_2502_20723_gb300 import synth
    (c0, m0), (c1, m1) = bench.replica_seeds(0), bench.replica_seeds(1)
    assert c0 != c1 and m0 != m1
    a = synth.random_configs(bench.N_SITES, 64, seed=c0)
    b = synth.random_configs(bench.N_SITES, 64, seed=c1)
    assert not np.array_equal(a[0], b[0])


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, device="cpu") == 3.5
    assert bench.replicas_rate(1, 3, 1.5) == pytest.approx(2.0)
