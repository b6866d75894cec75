"""Splitting orbits over ranks (one process per GPU).

Orbits are independent (the paper's embarrassingly parallel structure,
Sec. 1.2), and the Philox counter holds the GLOBAL orbit index, so a shard
integrated on its own produces bit for bit the orbits the unsharded run
produces.  There is no exchange step: the only collective is the benchmark's
max-over-ranks of the timed region.
"""


def shard(total_orbits, world_size, rank):
    """Contiguous share of rank: (orbit_offset, count); counts differ by at most 1."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("rank %d outside world of %d" % (rank, world_size))
    base, extra = divmod(int(total_orbits), int(world_size))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def weak_scaling_offset(orbits_per_rank, rank):
    """Global orbit index of a rank's first orbit when every rank runs the
    same per-GPU problem size (weak scaling)."""
    return int(rank) * int(orbits_per_rank)


def max_over_ranks(value, dist=None, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
