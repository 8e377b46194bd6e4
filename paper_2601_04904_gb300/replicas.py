"""Host-side logic of multi-GPU runs: independent energy-point replicas.

A single solve's sweep is sequential (Alg. 1 / Alg. 2), so GPUs only share
work at the level of independent energy points: one process per GPU, each
solving its own points, with no collective on the data path.  The only
communication is timing: a barrier around the timed region and the maximum of
the per-rank times, from which the whole-job rate is formed.  Everything here
is plain torch.distributed and runs on the gloo backend as well (CPU tests).
"""
from __future__ import annotations

import os

from . import inputs


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def energy_of(rank: int) -> float:
    """Energy of the point a rank solves: 0.3 (the benchmark's) on rank 0, the
    seeded grid E ~ U[-1, 1] elsewhere, so that replicas solve different
    points of the same device."""
    return 0.3 if rank == 0 else float(inputs.energy_grid(rank + 1)[0][rank])


def rhs_seed(rank: int) -> int:
    """Seed of the rank's lesser self-energy B (one per energy point)."""
    return inputs.BASE_SEED + 7 + rank


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """Maximum of a per-rank value (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, points_per_rank: int, seconds: float) -> float:
    """Whole-job energy points per second: every rank's points over the
    slowest rank's time (weak scaling: the per-rank work is fixed)."""
    return world * points_per_rank / seconds


def shard(n: int, rank: int, world: int) -> range:
    """Contiguous share of n independent items for a rank (sizes differ by at
    most one; the shares of all ranks partition range(n))."""
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))
