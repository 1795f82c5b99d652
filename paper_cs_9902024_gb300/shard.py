"""Runs sharded over processes, one per GPU.

The paper's first level of parallelism is the set of n statistically
independent runs (Sec. 1.3); across GPUs it needs no exchange while the runs
advance.  Rank k of N holds the runs with global indices k*n_k .. k*n_k +
n_k - 1 (``dsmc_options.run_offset``), so each run draws exactly the random
numbers it would draw in a one-process ensemble.  A run's moments go to
group (global run index) mod G, and the ensemble's group sums are the sums
over ranks of every rank's group sums -- one reduction per sample, after
the runs are done.  G = min(runs per rank, 16) must be the same on every
rank, so a sharded ensemble gives each rank at least 16 runs.
"""
from __future__ import annotations

import numpy as np

MAX_GROUPS = 16


def run_offset(rank: int, runs_per_rank: int) -> int:
    """Global index of a rank's first run."""
    return rank * runs_per_rank


def groups(runs_per_rank: int, world: int) -> int:
    """Batch-means group count of a sharded ensemble (the same on every
    rank)."""
    if world > 1 and runs_per_rank < MAX_GROUPS:
        raise ValueError("a sharded ensemble needs at least %d runs per rank" % MAX_GROUPS)
    return min(runs_per_rank, MAX_GROUPS)


def allreduce_group_sums(raws: np.ndarray) -> np.ndarray:
    """Sum the ranks' group sums (float64, any shape) with
    torch.distributed: on the GPU under NCCL, on the host under gloo."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(raws, dtype=np.float64))
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t)
    return t.cpu().numpy()


def allreduce_max(x: float) -> float:
    """Largest value over the ranks (e.g. a timed region's duration)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x: float) -> float:
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t)
    return float(t.item())
