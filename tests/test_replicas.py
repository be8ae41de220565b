"""Multi-GPU replicas: host logic on CPU with gloo, world size 2.

The GPU path runs one independent replica per rank (no data-path
collective); what ranks share is the timing reduction (the slowest rank
ends the job) and, for batched sets and serving requests, a contiguous
split of the items.  Both are exercised here in two gloo processes.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2510_09417_gb300.replicas import job_rate, shard_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    from paper_2510_09417_gb300.replicas import max_over_ranks, shard_range as sr
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        lo, hi = sr(4096, rank, ws)
        seconds = 1.5 + rank  # rank 1 is the slow one
        tmax = max_over_ranks(seconds)
        shares = [None] * ws
        dist.all_gather_object(shares, (lo, hi))
        q.put((rank, tmax, shares))
    finally:
        dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 7, 4096, 4097):
        for ws in (1, 2, 3, 8):
            got = [shard_range(n, r, ws) for r in range(ws)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def test_job_rate():
    assert job_rate(2e8, 4, 2.0) == pytest.approx(4e8)
    with pytest.raises(ValueError):
        job_rate(1.0, 1, 0.0)


def test_replicas_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, tmax, shares in out:
        assert tmax == pytest.approx(2.5)  # every rank sees the slowest rank's time
        assert shares == [(0, 2048), (2048, 4096)]
