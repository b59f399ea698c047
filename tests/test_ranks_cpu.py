"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1).

Under torchrun every rank answers its own query batch over its own index
replica (weak scaling, no data-path collective); the only exchange is the
MAX of the ranks' step times, and the job's rate is all ranks' queries over
that time.  The reference arm runs on rank 0 alone.
"""
import os
import socket

import numpy as np
import pytest

import bench
from paper_2407_03618_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))
    w = synth.WORKLOADS["tiny"]
    q = bench.rank_batch(w, rank, 16)
    sizes = torch.tensor([q.n_queries], dtype=torch.int64)
    dist.all_reduce(sizes)
    out[rank] = (ms, int(sizes.item()), q.tokens.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_the_slowest_time():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0          # the job's time is the slower rank's
    assert res[0][1] == res[1][1] == 32             # each rank its own 16 queries
    assert res[0][2] != res[1][2]                   # different batches (seed 1 + rank)
    assert bench.job_rate(16, world, 15.0) == pytest.approx(32 / 0.015)


def test_rank_batches_follow_the_workload_law():
    w = synth.WORKLOADS["tiny"]
    a, b = bench.rank_batch(w, 0), bench.rank_batch(w, 1)
    assert a.n_queries == b.n_queries == w.n_queries
    la, lb = np.diff(a.offsets), np.diff(b.offsets)
    assert la.min() >= 2 and lb.max() <= 8          # uniform 2..8 tokens
    assert np.array_equal(a.tokens, w.queries(seed=1).tokens)
    assert bench.max_over_ranks(12.5, 1, None) == 12.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.reference_arm(bench.parse()) == 0  # returns at once, no work
