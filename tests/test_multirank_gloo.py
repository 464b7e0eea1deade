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


# ---- independent solves sharded over ranks ---------------------------------
def test_partition_is_a_balanced_deterministic_cover():
    """Longest-processing-time assignment: disjoint, covers every item, the
    same on every call, and within Graham's 4/3 bound of the optimum (here
    checked against the trivial lower bound max(mean load, largest item))."""
    sys.path.insert(0, ROOT)
    from paper_2507_13754_gb300 import shard, workloads as W
    sizes = W.cfg4_grid_sizes()
    costs = [shard.solve_cost(n, 24) for n in sizes for _ in range(8)]  # 64 frequencies x 8 angles
    assert len(costs) == 512
    for world in (1, 2, 3, 8):
        shares = shard.partition(costs, world)
        assert shares == shard.partition(costs, world)
        flat = sorted(i for s in shares for i in s)
        assert flat == list(range(512))
        ld = shard.loads(costs, shares)
        lower = max(sum(costs) / world, max(costs))
        assert max(ld) <= 4.0 / 3.0 * lower + 1e-9, (world, max(ld) / lower)
    # more ranks than items: every item on its own rank, the rest idle
    assert shard.partition([5, 1, 3], 5) == [[0], [2], [1], [], []]
    assert shard.padded_size(2) == 16 and shard.padded_size(1024) == 2048 and shard.padded_size(1025) == 4096


def _shard_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2507_13754_gb300 import shard, workloads as W
    # cfg4: each rank derives its share of the 512 (frequency, angle) solves
    sizes = W.cfg4_grid_sizes()
    costs = [shard.solve_cost(n, 24) for n in sizes for _ in range(8)]
    mine = shard.partition(costs, world)[rank]
    # cfg5: the 16 sources split over the ranks; each rank's gradient is a
    # stand-in array per source (its index times a pattern), summed over its
    # share and then over the ranks
    src_costs = [shard.solve_cost(1024, 20)] * 16
    my_src = shard.partition(src_costs, world)[rank]
    pattern = torch.arange(12, dtype=torch.float64).reshape(3, 4)
    grad_c = sum((float(s + 1) * pattern for s in my_src), torch.zeros(3, 4, dtype=torch.float64))
    grad_a = sum((float(s + 1) ** 2 * pattern for s in my_src), torch.zeros(3, 4, dtype=torch.float64))
    shard.allreduce_sum_([grad_c, grad_a])
    dist.barrier()
    q.put((rank, mine, my_src, grad_c.tolist(), grad_a.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_sweep_and_sum_the_gradient():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (_, m0, s0, gc0, ga0), (_, m1, s1, gc1, ga1) = res
    assert not set(m0) & set(m1) and sorted(m0 + m1) == list(range(512))
    assert not set(s0) & set(s1) and sorted(s0 + s1) == list(range(16))
    pattern = torch.arange(12, dtype=torch.float64).reshape(3, 4)
    want_c = sum(float(s + 1) for s in range(16)) * pattern
    want_a = sum(float(s + 1) ** 2 for s in range(16)) * pattern
    for gc, ga in ((gc0, ga0), (gc1, ga1)):
        assert torch.equal(torch.tensor(gc, dtype=torch.float64), want_c)
        assert torch.equal(torch.tensor(ga, dtype=torch.float64), want_a)
