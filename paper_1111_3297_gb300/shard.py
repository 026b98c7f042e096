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
