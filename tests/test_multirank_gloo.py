"""Multi-process (world size 2, gloo on CPU) checks of the benchmark's rank
bookkeeping: each rank solves its own replica, the job time is the slowest
rank's, and the job rate counts every rank's updates (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        elapsed = 2.0 + rank          # rank 1 is the slow one
        t = bench.max_over_ranks(elapsed)
        value = bench.job_throughput(1e6, world, t)
        # replicas differ by seed but share the workload shape
        w = bench._workload(_Args(), seed=rank)
        q.put((rank, t, value, w.nx, w.ny, float(w.fibers[0, 0])))
    finally:
        dist.destroy_process_group()


class _Args:
    nx, ny, fibers_per_band = 1152, 256, 10


def test_two_rank_max_time_and_weak_scaling():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, value, nx, ny, x0 in out:
        assert t == 3.0                       # max over ranks
        assert value == pytest.approx(1e6 * 2 / 3.0 * 1e-6)
        assert (nx, ny) == (1152, 256)
    assert out[0][5] != out[1][5]             # different seeds per replica


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.job_throughput(3e6, 1, 2.0) == pytest.approx(1.5)
