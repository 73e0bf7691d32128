"""Work split across ranks, on CPU: instance partition, the timing
reduction under torch.distributed with the gloo backend at world size 2,
and a sharded batch stepped by two ranks (the FP64 oracle standing in for
the GPU step, which needs a device) against the same batch in one
process."""
import os

import pytest

from paper_2510_25702_gb300 import cases
from paper_2510_25702_gb300.shard import combine_timing, partition_instances, shard_cases


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


def _small_batch():
    return cases.batched_channels(n_instances=5, dps=(0.1,), seed=5)


def _fingerprint(case, steps):
    from oracle import OracleSim

    o = OracleSim(case)
    o.step(steps)
    f = o.fields()
    return {k: f[k].copy() for k in ("uid", "pos", "vel", "rho")}


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    batch = _small_batch()
    names = [c.name for c in batch]
    mine = shard_cases(batch, world, rank)
    res = {names.index(c.name): _fingerprint(c, 3) for c in mine}
    # the results meet on rank 0 only for the check (the step itself has no
    # data-path collective)
    got = [None] * world if rank == 0 else None
    dist.gather_object(res, got, dst=0)
    if rank == 0:
        merged = {}
        for part in got:
            for q, f in part.items():
                assert q not in merged, "instance stepped by two ranks"
                merged[q] = f
        out["merged"] = merged
    ms, ps = combine_timing(1.0 + rank, float(sum(c.n for c in mine)), dist)
    out[rank] = (ms, ps)
    dist.destroy_process_group()


def test_sharded_batch_matches_one_process_gloo_world2(orc):
    mp = pytest.importorskip("torch.multiprocessing")
    import socket

    import numpy as np

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    batch = _small_batch()
    merged = out["merged"]
    assert sorted(merged) == list(range(len(batch)))
    for q, c in enumerate(batch):
        ref = _fingerprint(c, 3)
        for k in ref:
            assert np.array_equal(merged[q][k], ref[k]), (q, k)
    total = float(sum(c.n for c in batch))
    assert out[0] == out[1] == (2.0, total)
