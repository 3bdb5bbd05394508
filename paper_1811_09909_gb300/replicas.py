"""Host logic of multi-GPU runs: the path does not shard within one problem,
so N GPUs run N independent replicas (one process per GPU, launched by
torch.distributed.run).  Each rank solves its own seeded problem (or its share
of a batch of independent problems); the time of a step is the maximum over
ranks, and the whole-job rate counts every rank's units.  No data-path
collective exists; the only collectives are a barrier and one MAX reduction
of the timings."""
import os


def rank_info():
    """(rank, world size, local rank) from the torch.distributed.run environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_units, rank, world):
    """Contiguous, balanced share [lo, hi) of n_units independent units for one
    rank: the shares of all ranks cover every unit exactly once and differ by
    at most one unit."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def replica_seed(seed, rank):
    """Seed of rank's replica: distinct per rank, rank 0 keeps the base seed."""
    return seed + 1000 * rank


def max_over_ranks(value, dist=None, device=None):
    """The maximum of a float over all ranks (the value itself without a
    process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_ms):
    """Units processed by all ranks per second, over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)
