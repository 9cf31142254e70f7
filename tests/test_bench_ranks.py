"""The benchmark's multi-rank path on CPU (two gloo processes): every rank
gets the slowest rank's step time, and the job's value counts the bytes of
all ranks over that time (replicas, no collective on the data path)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [2.5, 7.25][rank]
    got = bench.max_over_ranks(ms, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, bench.job_value(world, 16_000_000, got)))


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [7.25, 7.25]
    assert res[0][2] == pytest.approx(2 * 16_000_000 / 7.25e-3 / 1e9)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_value(1, 16e6, 0.25) == pytest.approx(64.0)
