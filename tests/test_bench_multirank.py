"""The benchmark's multi-rank host logic (independent replicas, one barrier,
the slowest rank's time) with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # rank r took (r + 1) * 10 ms for the same per-rank work
    value, ms = bench.whole_job(w, 1000.0, 10.0 * (rank + 1))
    out.put((rank, value, ms))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_replicas_report_whole_job_throughput_at_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == 20.0                       # max over ranks
        assert value == pytest.approx(2 * 1000.0 / 0.020)   # both ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.whole_job(1, 500.0, 5.0) == (pytest.approx(1e5), 5.0)
