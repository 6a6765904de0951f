"""The multi-GPU path of this repository is replicas only: every rank builds
and samples its own table and the bench combines timings across ranks (max
of the per-rank times, work summed).  This CPU test runs that combination
with world size 2 over gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r pretends its build took 10 + r ms and its sampling 20 - r ms
    tb, ts = bench.reduce_max([10.0 + rank, 20.0 - rank], "cpu")
    rates = bench.job_rates(world, 3, 1000, 2000, tb, ts)
    q.put((rank, tb, ts, rates))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine_by_slowest_rank():
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
    for rank, tb, ts, (gw, gs) in out:
        assert tb == 11.0 and ts == 20.0  # max over both ranks, identical on each
        assert gw == pytest.approx(2 * 3 * 1000 / 11e-3 / 1e9)
        assert gs == pytest.approx(2 * 3 * 2000 / 20e-3 / 1e9)


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_max([1.5, 2.5], "cpu") == [1.5, 2.5]
    assert bench.job_rates(1, 2, 10, 20, 1.0, 2.0) == pytest.approx((2e-5, 2e-5))
