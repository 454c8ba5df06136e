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


# ---------------------------------------------------------------------------
# Liveness between steps
#
# A rank that raised, exited or never joined is found on the host, through a
# key-value store the ranks share (any torch.distributed Store: the process
# group's TCPStore, a FileStore), before the next launch or collective:
# every rank records each step it finished, and before starting the next one
# waits, with a short limit, until every other rank has recorded it.  The
# surviving ranks then learn which ranks were lost instead of waiting inside
# a collective for a peer that will never arrive; their own chains and
# results are untouched.
# ---------------------------------------------------------------------------


class PeerLost(RuntimeError):
    """Ranks that did not record a step within the liveness limit."""

    def __init__(self, step: int, ranks):
        self.step = int(step)
        self.ranks = sorted(int(r) for r in ranks)
        super().__init__("rank(s) %s did not finish step %d" % (", ".join(map(str, self.ranks)), self.step))


def _step_key(step: int, rank: int) -> str:
    return "tl/step/%d/%d" % (step, rank)


def heartbeat(store, rank: int, step: int) -> None:
    """Record in `store` that `rank` finished `step`: its work for the step is
    complete and nothing of it is still in flight."""
    store.set(_step_key(step, rank), b"1")


def wait_peers(store, world: int, step: int, timeout_s: float, poll_s: float = 0.01) -> None:
    """Return once every rank of `world` has recorded `step`; raise PeerLost
    naming the ranks that have not after `timeout_s` seconds."""
    import time
    keys = [_step_key(step, r) for r in range(world)]
    deadline = time.monotonic() + float(timeout_s)
    while True:
        missing = [r for r, k in enumerate(keys) if not store.check([k])]
        if not missing:
            return
        if time.monotonic() >= deadline:
            raise PeerLost(step, missing)
        time.sleep(poll_s)
