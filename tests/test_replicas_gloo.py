"""Host logic of the multi-GPU layout, which is replicas only: every rank
decodes and renders its own copy of the workload with no collective on the
data path, and the job's time is the slowest rank's.  Run as two gloo ranks
on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r is slower by r ms; every rank must see the maximum
        mine = [10.0 + rank, 3.0 - rank, 7.0]
        got = bench.max_over_ranks(mine, world, "cpu")
        dist.barrier()
        q.put((rank, got, bench.job_mpix_per_s(world, 1_000_000, got[0])))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in procs:
        r, got, v = q.get(timeout=120)
        out[r] = (got, v)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        got, v = out[r]
        assert got == [11.0, 3.0, 7.0]
        # 2 replicas x 1 Mpx in 11 ms
        assert v == pytest.approx(2 * 1e6 / 11e-3 / 1e6)


def test_one_rank_is_the_identity():
    assert bench.max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]
    assert bench.job_mpix_per_s(1, 2_000_000, 4.0) == pytest.approx(500.0)
