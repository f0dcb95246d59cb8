"""Multi-rank bookkeeping of the benchmark on the CPU (two gloo ranks): each
rank gets its own independent room seed, the step time is the slowest rank's,
and the job value counts every rank's pairs.  No GPU and no data-path
collective are involved (the path partitions into independent rooms)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds("ward", rank)
        ms = [120.0, 150.0][rank]                  # the second rank is slower
        slowest = bench.max_over_ranks(ms, dist, "cpu")
        dist.barrier()
        out[rank] = (seeds, slowest, bench.job_value(2_000_000, world, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == (1, 2) and res[1][0] == (1001, 1002)      # independent rooms
    assert res[0][1] == res[1][1] == 150.0                          # max over ranks
    assert res[0][2] == pytest.approx(2 * 2_000_000 / 0.150 / 1e9)  # whole-job pairs/s


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.rank_seeds("large", 0) == (3, 2)
