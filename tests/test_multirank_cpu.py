"""The multi-rank paths of bench.py (independent replicas, weak scaling) on
two gloo ranks on the CPU: barrier, max over ranks, whole-job throughput."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    assert bench.dist_env() == (world, rank, rank)
    bench.dist_barrier()
    m = bench.dist_max(1.5 + rank)
    value, t = bench.weak_scaling_value(units_per_rank=1000.0, seconds_this_rank=2.0 + rank)
    q.put((rank, m, value, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    for rank, m, value, t in out:
        assert m == 2.5
        assert t == 3.0
        assert value == pytest.approx(2 * 1000.0 / 3.0)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.dist_max(4.25) == 4.25
    assert bench.weak_scaling_value(10.0, 2.0) == (5.0, 2.0)
