"""The bench's multi-rank host logic on two gloo ranks (CPU).

Weak scaling: every rank takes its own consecutive blocks of atoms, the timed region is closed by a
barrier, the job time is the slowest rank's, and the whole-job throughput counts the columns of all
ranks. Two processes run the bench's own functions over a gloo process group (127.0.0.1).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import importlib.util
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
        bench = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(bench)
        N, B, warmup, steps = 1000, 64, 2, 3
        mine = np.concatenate([bench.shard_atoms(rank, i, warmup + steps, B, N) for i in range(warmup + steps)])
        got = [None] * world
        dist.all_gather_object(got, mine.tolist())
        ms = 100.0 + 50.0 * rank               # the ranks' own timed-region lengths
        bench.rank_barrier()
        mx = bench.max_over_ranks(ms)
        val = bench.job_throughput(4 * B, steps, world, mx)
        out[rank] = (got, mx, val)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_disjointly_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    shards0, mx0, val0 = res[0]
    shards1, mx1, val1 = res[1]
    assert shards0 == shards1                                  # both ranks see the same assignment
    a, b = set(shards0[0]), set(shards0[1])
    assert len(a) == len(shards0[0]) and len(b) == len(shards0[1])
    assert not (a & b)                                          # no atom on two ranks
    assert mx0 == mx1 == 150.0                                  # the slowest rank's time
    assert val0 == val1 == pytest.approx(4 * 64 * 3 * 2 / 0.150)
