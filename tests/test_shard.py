"""Work split across ranks, on CPU: instance partition and the timing
reduction under torch.distributed with the gloo backend, world size 2."""
import os

import pytest

from paper_2510_25702_gb300 import cases
from paper_2510_25702_gb300.shard import combine_timing, partition_instances


def test_partition_covers_every_instance_once_and_balances():
    counts = [c.n for c in cases.batched_channels()]
    for world in (1, 2, 3, 8):
        parts = partition_instances(counts, world)
        flat = sorted(q for p in parts for q in p)
        assert flat == list(range(len(counts)))
        loads = [sum(counts[q] for q in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean by more than the largest instance
        assert max(loads) - sum(loads) / world <= max(counts)


def test_partition_more_ranks_than_instances():
    parts = partition_instances([5, 3], 4)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts = [c.n for c in cases.batched_channels()]
    mine = partition_instances(counts, world)[rank]
    ms = 10.0 + rank  # rank 1 is the slower one
    ps = float(sum(counts[q] for q in mine))
    out[rank] = combine_timing(ms, ps, dist)
    dist.destroy_process_group()


def test_combine_timing_gloo_world2():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    total = float(sum(c.n for c in cases.batched_channels()))
    for r in range(2):
        ms, ps = out[r]
        assert ms == 11.0 and ps == total
