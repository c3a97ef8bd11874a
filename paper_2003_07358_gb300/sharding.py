"""Host-side sharding of independent spectral sub-problems across GPUs.

The faceted problem splits into independent channel-interleaved sub-cubes
(Section 2.4.1): there is no exchange between them, so the natural multi-GPU
layout is one process per GPU, each owning whole cubes, with no data-path
collective.  Ranks only meet at barriers and at the end (max of the step times
for the benchmark; gather of results if a caller wants them).

Two policies:
  * replicate_cubes: every rank runs the full workload on its own seeded cube
    (weak scaling: per-GPU work fixed as the number of GPUs grows);
  * split_subcubes: the C sub-cubes of one cube are dealt round-robin to ranks
    (strong scaling of a single cube).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info(env=None) -> RankInfo:
    env = os.environ if env is None else env
    return RankInfo(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))


def replicate_cubes(n_subcubes: int, info: RankInfo) -> tuple[int, list[int]]:
    """(seed offset, sub-cubes) of this rank when every rank owns a full cube."""
    return info.rank, list(range(n_subcubes))


def split_subcubes(n_subcubes: int, info: RankInfo) -> list[int]:
    """Sub-cubes of this rank when one cube's sub-cubes are dealt round-robin."""
    return [c for c in range(n_subcubes) if c % info.world == info.rank]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank time over the process group (identity without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return units_per_rank * world / seconds_max
