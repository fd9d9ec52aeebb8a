"""Bookkeeping of runs on several GPUs of one node (one process per GPU).

The per-step path does not shard: every rank steps its own independent tank
(weak scaling) and no collective touches the data path.  Only the timing is
combined: the slowest rank's time of the timed region counts, and the
throughput counts the nodes of every rank.
"""
import os


def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class RankFailure(RuntimeError):
    """A peer rank did not reach a collective in time (it failed or left)."""


def init_process_group(backend, timeout_s=600.0, **kw):
    """torch.distributed's process group with a bounded wait on every
    collective: a rank that fails or leaves makes the others' next barrier
    or reduction raise instead of waiting forever."""
    import datetime
    import torch.distributed as dist
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s), **kw)


def barrier(world):
    """Wait for every rank; RankFailure if a peer does not arrive within the
    process group's timeout (or has gone)."""
    if world > 1:
        import torch.distributed as dist
        try:
            dist.barrier()
        except RuntimeError as e:
            raise RankFailure("a rank did not reach the barrier: %s" % str(e).splitlines()[0]) from e


def max_over_ranks(value, world, device=None):
    """The maximum of a float over all ranks (the value itself on one rank).
    device: where the reduction tensor lives (a CUDA device for NCCL, None
    for CPU backends such as gloo)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank, world, ms_max):
    """Units per second of the whole job: every rank's units over the slowest
    rank's time (milliseconds)."""
    return units_per_rank * world / (ms_max * 1e-3)
