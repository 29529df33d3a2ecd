"""Batch sharding over ranks, one GPU per rank.

The instances of a batch are independent Couette problems (each is solved on its own
grid and velocity set, Sec. II), so splitting the instance list over ranks needs no
collective on the data path: every rank builds a Solver over its share and steps it
alone. Only the per-instance results (steps taken, residuals, profiles) travel, on the
host, once a run is over.

    idx = shard(instances, rank, world)
    s = Solver([instances[i] for i in idx], ...)
    ...
    steps = gather(list_of_local_results, idx, len(instances), dist)  # global order
"""


def cost(inst):
    """Cell x velocity updates per RK step of one instance (Nz Q), the unit of work."""
    return inst.Nz * inst.Q


def partition(instances, world, weight=cost):
    """Split the instance indices over world ranks, balancing the work per step.

    Longest-processing-time rule: instances by decreasing weight (ties by index), each to
    the rank with the least work so far (ties to the lower rank). No rank carries more
    than the mean plus the largest single instance. Returns world lists of indices, each
    ascending. The result depends only on the weights and world, so every rank computes
    the same partition without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = [int(weight(i)) for i in instances]
    load = [0] * world
    parts = [[] for _ in range(world)]
    for b in sorted(range(len(w)), key=lambda b: (-w[b], b)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(b)
        load[r] += w[b]
    return [sorted(p) for p in parts]


def shard(instances, rank, world, weight=cost):
    """The indices of the instances rank owns, ascending (see partition)."""
    if not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return partition(instances, world, weight)[rank]


def gather(local, indices, n, dist=None):
    """Per-instance results of every rank, in global instance order, on every rank.

    local[k] is the result of global instance indices[k] on this rank. With dist (an
    initialised torch.distributed) the ranks exchange their lists as Python objects on
    the host; without it the call is the single-rank case. Raises if the ranks' indices
    do not cover 0 .. n-1 exactly once."""
    if len(local) != len(indices):
        raise ValueError("one result per owned index")
    pairs = [list(zip(indices, local))]
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        pairs = [None] * dist.get_world_size()
        dist.all_gather_object(pairs, list(zip(indices, local)))
    out = [None] * n
    seen = [False] * n
    for part in pairs:
        for i, v in part:
            if not 0 <= i < n or seen[i]:
                raise ValueError("instance %d owned twice or out of range" % i)
            seen[i] = True
            out[i] = v
    if not all(seen):
        raise ValueError("instances %s owned by no rank" % [i for i in range(n) if not seen[i]])
    return out
