"""The multi-rank host logic of the benchmark on CPU: two gloo ranks agree on the slowest
rank's time and on the whole-job throughput (replicas, no collective in the data path)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    slowest = bench.max_over_ranks(ms, world)
    q.put((rank, slowest, bench.job_throughput(4 * 23.59e6, world, 10, slowest)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    expect = 4 * 23.59e6 * 2 * 10 / 1e6 / (20.0 / 1e3)
    assert all(abs(o[2] - expect) < 1e-9 * expect for o in out)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.job_throughput(1e6, 1, 1, 1000.0) == pytest.approx(1.0)
