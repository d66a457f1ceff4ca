"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) take the
slowest rank's time, and the whole-job throughput counts every rank's nodes."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 95.0][rank]
    worst = bench.max_over_ranks(local_ms, dist, device="cpu")
    dist.barrier()
    out.put((rank, worst, bench.job_mlups(world, 1000, 10, worst / 1e3)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [120.0, 120.0]
    # 2 ranks x 1000 nodes x 10 steps in 0.12 s
    assert all(abs(g[2] - 2 * 1000 * 10 / 0.12 / 1e6) < 1e-12 for g in got)


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_mlups(1, 512 ** 3, 20, 0.1516) == pytest.approx(512 ** 3 * 20 / 0.1516 / 1e6)
