"""The replica (N > 1) path of bench.py on CPU: two gloo ranks each report
their own device time and Born-term units; the job's value is the summed units
over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [0.5, 0.8][rank]
    units = [1000, 3000][rank]
    t_max, u = bench.aggregate_ranks(t, units, world, "cpu")
    dist.barrier()
    q.put((rank, t_max, u))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_driver():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, u in res:
        assert t_max == 0.8 and u == 4000.0
    assert 4000.0 / 0.8 == 5000.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(0.25, 10, 1, "cpu") == (0.25, 10.0)
