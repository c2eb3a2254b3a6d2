"""The benchmark's multi-rank path on the CPU: two gloo ranks (the replicas
the benchmark runs one per GPU) agree on the slowest rank's time, and the
job's rate counts every rank's units over that time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(1.5 + rank, "cpu")
        dist.barrier()
        out.put((rank, ms, bench.job_rate(ws, 1000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [ms for _, ms, _ in res] == [2.5, 2.5]
    assert all(rate == 2 * 1000 / 2.5e-3 for _, _, rate in res)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25
    assert bench.job_rate(1, 50, 2.0) == 25000.0
