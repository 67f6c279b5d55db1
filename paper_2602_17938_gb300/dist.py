"""Frame sharding across ranks (one process per GPU): no data-path collective.

Frames are independent, so N ranks clean N disjoint sets of frames (weak
scaling).  The only cross-rank step is reporting: the job's time is the
maximum over ranks, and its throughput is the pixels of all ranks divided
by that time.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def frames_for_rank(n_frames: int, rank: int, world: int) -> list[int]:
    """Round-robin assignment of frame indices to ranks (disjoint, covering)."""
    return list(range(rank, n_frames, world))


def frame_seed(config_seed: int, rank: int) -> tuple:
    """Seed of the frame a rank cleans in the single-frame benchmark."""
    return (config_seed, rank)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (a time) over the process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pixels_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job Mpix/s: every rank's pixels over the slowest rank's time."""
    return world * pixels_per_rank * steps / 1e6 / max_seconds
