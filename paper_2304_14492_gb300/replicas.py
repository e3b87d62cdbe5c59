"""Host-side plumbing of multi-GPU runs: images are independent, so N GPUs run
N replicas of the whole path, one process per GPU, each on its own disjoint
shard of frames, with no collective on the data path.  The only collectives
are a barrier before the timed region and the maximum of the ranks' times
after it (the job is as slow as its slowest rank)."""

import os


def dist_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard(rank, per_rank):
    """Frame indices of one rank: disjoint, contiguous shards of `per_rank`."""
    return range(rank * per_rank, (rank + 1) * per_rank)


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks (the value itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, per_rank, steps, ms):
    """Units processed by all ranks per second, given the slowest rank's time."""
    return world * per_rank * steps / (ms / 1000.0)
