"""Several GPUs as independent replicas: one process per GPU, no collective on
the data path.

Independent chains, batches of chains and request streams split by job: rank
r of N takes every N-th job and keys its random numbers by the job's own
stream id, so a job's result does not depend on which rank ran it.  Only the
timing (the slowest rank's) and the per-job results meet on the host at the
end, through torch.distributed (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Jobs of rank `rank`: every world-th item starting at `rank`."""
    if not 0 <= rank < world:
        raise ValueError("rank %d outside world of %d" % (rank, world))
    return list(items)[rank::world]


def replica_stream_id(base: int, rank: int, world: int) -> int:
    """Stream id of replica `rank` of a workload whose single-GPU stream id is
    `base`: distinct for every (base, rank), equal to `base` on one GPU."""
    return base * world + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's wall time is the slowest
    rank's).  Without a process group, the value itself."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(obj, dist=None) -> list:
    """Every rank's `obj`, in rank order (a list of one without a group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
