"""One process per GPU: walker sharding with no data-path collective.

The walkers of a Monte Carlo run are independent Markov chains: every
determinant or Pfaffian update touches one walker's own matrices only, so the
batch splits across GPUs as whole walkers.  Each rank draws its own shard of
walkers from a rank-shifted seed and advances it with no exchange; the only
collectives are on the host side of a measurement: a barrier around the timed
region and a MAX of the per-rank elapsed times (the job takes as long as its
slowest rank).  The whole-job rate is then the units of all ranks over that
time (weak scaling: the per-rank shard is fixed as ranks are added).
"""
import os

SEED_STRIDE = 1000   # rank r draws its shard from seed + r * SEED_STRIDE


def rank_env():
    """(rank, world, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed(seed, rank):
    """Seed of rank `rank`'s walker shard; rank 0 keeps the single-process seed."""
    return seed + SEED_STRIDE * rank


def max_over_ranks(value, dist=None, device="cpu"):
    """Maximum of a per-rank float over all ranks (the value itself without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank, world, ms_max):
    """Units of all ranks per second, timed by the slowest rank."""
    return units_per_rank * world / (ms_max / 1e3)
