"""Interval sharding across ranks (one process per GPU).

Segments are independent given their first hits (Lemma lem:q applied at f+t), so
an interval splits into contiguous runs of segments with no exchange during
sieving.  Weak scaling gives every rank its own n segments (rank r sieves
f + r*n .. f + (r+1)*n); strong scaling splits one interval of n segments.
The only collective is a host-side sum of composite counts.
"""


def shard(l, f, n, rank, world, scaling="weak"):
    """(f_r, n_r) of rank `rank` among `world` ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    if scaling == "weak":
        return f + rank * n, n
    if scaling == "strong":
        base, extra = divmod(n, world)
        start = rank * base + min(rank, extra)
        return f + start, base + (1 if rank < extra else 0)
    raise ValueError("scaling must be 'weak' or 'strong'")


def total_count(local_count, group=None):
    """Sum of the ranks' composite counts (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(local_count)], dtype=torch.int64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())


def request_cost(j0, nbits):
    """Estimated device work of one request (j0, nbits): its bits, plus a first-hit
    visit per base prime up to the root of its last number (x / ln x primes below
    x), which dominates short requests of high magnitude."""
    import math
    root = math.isqrt(2 * (j0 + nbits - 1) + 1)
    return nbits + 8.0 * root / max(1.0, math.log(max(root, 3)))


def partition_requests(reqs, rank, world):
    """Indices (ascending) of the requests (j0, nbits) that rank `rank` of `world`
    serves: the batch and serving forms run replicas, one per GPU, each on its own
    share.  Longest-processing-time first: requests in order of decreasing cost go to
    the rank with the least assigned cost so far (ties to the lower rank), so every
    rank computes the same partition without communicating, the shares are disjoint,
    cover every request, and their costs differ by at most the largest request's."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    costs = [request_cost(j0, nb) for j0, nb in reqs]
    order = sorted(range(len(reqs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)
