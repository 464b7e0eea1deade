"""Independent solves spread over ranks (one process per GPU).

One field does not shard: splitting a 2D FFT over GPUs needs two all-to-all
transposes per Born term, about as many bytes over the interconnect as the
term moves through HBM.  Independent solves do shard: the frequencies and
steering angles of a broadband sweep, or the sources of a gradient
evaluation, run on different GPUs with nothing exchanged during the forward
series.  The gradient of a misfit summed over sources needs one sum over
ranks of grad_c and grad_alpha at the end (``allreduce_sum_``).

The unit of work is one solve (one right-hand side on one grid).  Its cost is
taken as M^2 * terms, M the padded FFT size: a Born term moves ~92 N^2 =
23 M^2 bytes, so the cost is proportional to HBM traffic.  ``partition``
assigns solves to ranks by the longest-processing-time rule (largest first,
each to the least-loaded rank), deterministically, so that every rank
computes the same assignment without communicating.
"""
from __future__ import annotations

import heapq


def padded_size(n: int) -> int:
    """The library's FFT size for an N x N grid: the smallest power of two
    >= max(2N - 1, 16) (zero padding for the linear convolution)."""
    m = 16
    while m < 2 * n - 1:
        m *= 2
    return m


def solve_cost(n: int, terms: int) -> int:
    """Cost of one solve: M^2 * terms (proportional to its HBM traffic)."""
    return padded_size(n) ** 2 * int(terms)


def partition(costs, world: int):
    """Assign item i (cost costs[i]) to one of `world` ranks.

    Largest cost first (ties: lower index first), each to the rank with the
    least load so far (ties: lower rank).  Returns a list of `world` sorted
    index lists; their union is range(len(costs)) and they are disjoint.
    The heaviest rank carries at most 4/3 of the optimal makespan (Graham's
    bound for this rule)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def loads(costs, shares):
    """Total cost per rank of a partition."""
    return [sum(costs[i] for i in s) for s in shares]


def sweep_solves(workloads, terms=None):
    """The solves of a sweep given as Workloads with n_rhs right-hand sides
    each (cfg4: one per frequency, one RHS per steering angle): a list of
    (workload index, rhs index) and their costs."""
    items, costs = [], []
    for k, w in enumerate(workloads):
        t = w.max_terms if terms is None else terms
        for r in range(w.n_rhs):
            items.append((k, r))
            costs.append(solve_cost(w.n, t))
    return items, costs


def rank_solves(workloads, world: int, rank: int, terms=None):
    """This rank's solves of a sweep, grouped by workload: {workload index:
    [rhs indices]} (each group becomes one plan with that many RHS)."""
    items, costs = sweep_solves(workloads, terms)
    mine = partition(costs, world)[rank]
    out = {}
    for i in mine:
        k, r = items[i]
        out.setdefault(k, []).append(r)
    return out


def allreduce_sum_(tensors, group=None):
    """Sum each tensor over the ranks of `group` in place (a no-op without an
    initialised process group or with one rank).  Used for grad_c and
    grad_alpha of a misfit summed over sources that ranks split."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return tensors
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors
