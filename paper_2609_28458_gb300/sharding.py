"""Ensemble sharding across processes, one GPU per process.

Members of an ensemble are independent (Sec. 2.1, Eq. ivp), so a shard is a contiguous range of
members and no data moves between ranks while solving. For parameters shared by every member, the
gradient of a loss summed over members is the sum of the per-member gradients (Appendix A,
Eq. chain): summed within a rank, then across ranks with one all-reduce of a p-vector.
"""
import torch


def shard_bounds(n_total, world, rank):
    """[start, stop) of rank's contiguous share of n_total members; sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad shard request: n=%d world=%d rank=%d" % (n_total, world, rank))
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def sum_shared_gradient(per_member, group=None):
    """Sum of per-member parameter gradients [n, p] over the members of this rank and, when a
    process group is initialised, over all ranks. Returns a p-vector on every rank."""
    local = per_member.sum(dim=0)
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(local, op=dist.ReduceOp.SUM, group=group)
    return local
