"""The multi-process (torchrun) path of bench.py on CPU with the gloo backend,
world size 2: per-rank image shards differ, the job time is the maximum over
ranks, and the throughput counts every rank's units (weak scaling)."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


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
    import bench
    from workloads import make_workload
    wl = make_workload("n32_tiny", seed=bench.rank_seed(rank), n_images=2, n_templates=2)
    t = bench.max_over_ranks(1.0 + rank, world, torch.device("cpu"))
    v = bench.job_throughput(100.0, 3, world, t)
    dist.barrier()
    q.put((rank, t, v, float(wl.images.sum())))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, s0), (r1, t1, v1, s1) = res
    assert t0 == t1 == 2.0               # the slowest rank's time
    assert v0 == v1 == 2 * 100.0 * 3 / 2.0
    assert s0 != s1                       # different image shards


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_throughput(10.0, 2, 1, 4.0) == 5.0
