"""Sharding over ranks, one GPU each: the batched form's problems, and the
plan for sharding one solve's tile pairs.

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


def partition_tile_pairs(np_, world, tile=32):
    """The plan for sharding one solve over `world` ranks (each RK stage: every
    rank holds the whole stage input, forms X_IJ = H_I. Y_.J and X_JI for its
    tile pairs (I, J), I <= J, of `tile` x `tile` tiles of the padded edge
    np_, writes tiles (I, J) and (J, I) of the next stage input, and the ranks
    exchange those tiles (an all-gather) and add their trace and residual
    partials (an all-reduce)). Pairs are dealt longest first to the least
    loaded rank, an off-diagonal pair costing twice a diagonal one (two tiles
    of products and of outputs). Returns, per rank, its list of (I, J)."""
    nt = (np_ + tile - 1) // tile
    pairs = [(i, j) for i in range(nt) for j in range(i, nt)]
    costs = [1.0 if i == j else 2.0 for i, j in pairs]
    return [[pairs[k] for k in part] for part in partition(costs, world)]


def stage_exchange_bytes(np_, world, tile=32, element_bytes=8):
    """Bytes each rank receives per RK stage in the plan above: the tiles the
    other ranks wrote (element_bytes per complex element: 8 for the FP32
    delta planes of the mixed form)."""
    parts = partition_tile_pairs(np_, world, tile)
    tiles = [sum(1 if i == j else 2 for i, j in p) for p in parts]
    total = sum(tiles)
    return [(total - t) * tile * tile * element_bytes for t in tiles]
