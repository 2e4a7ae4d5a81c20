"""Sharding the batched form over ranks, one GPU each.

The problems of a batch are independent (each its own graph, omega and
state, integrated to its own residual), so rank r solves a subset of them
with qpr_batch_steady_state and nothing is exchanged on the data path; the
batch is done when the slowest rank is. The subsets balance an estimate of
each problem's work: N^2 elements per stage times a step count that grows
as the dissipative part weakens (the spectral gap of the Lindblad
superoperator shrinks roughly with omega on these graphs), i.e. N^2 / omega.
"""


def batch_cost(n, omega):
    """Estimated work of one problem of size n at mixing omega."""
    return float(n) * float(n) / max(float(omega), 0.05)


def partition(costs, world):
    """Indices of the problems of each of `world` ranks: longest processing
    time first (costs in decreasing order, ties by index), each to the rank
    with the least assigned cost (ties: the lowest rank). Every index is in
    exactly one list; each list is in increasing order. The largest load is
    at most the mean load plus the largest cost."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]
