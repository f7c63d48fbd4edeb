"""Host-side logic of a Monte-Carlo run spread over ranks (one process per
GPU): which block of trials a rank draws, how per-rank statistics and
timings combine, and the whole-job throughput.  The trials of different ranks
are independent, so the data path needs no collective; only these few scalars
cross ranks (through whatever process group the caller initialised: NCCL on
GPUs, gloo in the CPU tests)."""
from __future__ import annotations

import numpy as np


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s block of trials (weak scaling: every rank draws its
    own trials, rank 0's are the single-GPU run's)."""
    return int(seed) + 1000 * int(rank)


def merge_stats(stats) -> np.ndarray:
    """Combine per-rank {mean, M2, count} (the layout of xlmimo_sumrate's
    `stats`) into the statistics of the union, by the pairwise update of Chan,
    Golub and LeVeque, in rank order."""
    mean, m2, n = 0.0, 0.0, 0.0
    for s in stats:
        mb, m2b, nb = float(s[0]), float(s[1]), float(s[2])
        if nb == 0:
            continue
        tot = n + nb
        d = mb - mean
        mean += d * nb / tot
        m2 += m2b + d * d * n * nb / tot
        n = tot
    return np.array([mean, m2, n])


def allgather_stats(stats, dist) -> np.ndarray:
    """merge_stats over every rank of the default process group."""
    import torch
    world = dist.get_world_size()
    t = torch.as_tensor(np.asarray(stats, np.float64).reshape(3))
    parts = [torch.zeros(3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, t.cpu())
    return merge_stats([p.numpy() for p in parts])


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world: int, trials_per_rank: int, steps: int, total_ms: float) -> float:
    """Whole-job trials per second: every rank's trials over the slowest rank's time."""
    return world * trials_per_rank * steps / (total_ms / 1e3)
