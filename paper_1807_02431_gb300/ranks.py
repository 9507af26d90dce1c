"""Host logic for running the method on several GPUs, one process per GPU (torch.distributed).

Replicas are independent between exit tests (Section 2.4), so a run shards by contiguous replica ranges.
The exchanges per exit test are small (Section 2.4.1 and 2.4.2):
  * the first exit of the parallel step: a MIN all-reduce of the packed key (check M << 32 | replica k),
    where k is the global replica index, so the lowest index wins at equal M as in Eq. 5;
  * the Gelman-Rubin sums of Eq. 3: a SUM all-reduce of (sum of replica means, sum of squared replica
    means, sum of within-replica variances, replica count) per observable;
  * the benchmark's wall time: a MAX all-reduce.
Independent replica sets per rank (the benchmark's "replicas only" mode) need only the last one.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

NO_EXIT = (1 << 64) - 1


def rank_seed(seed: int, rank: int) -> int:
    """Philox key of rank `rank` for independent replica sets (distinct noise streams per rank)."""
    return seed + 1000 * rank


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous replica range (start, count) of `rank`; the first n_total % world ranks take one more."""
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def first_exit(local_key: int, start: int, group=None, device=None) -> tuple[int, int] | None:
    """Global first exit from this rank's local key ((M << 32) | local replica, or NO_EXIT).

    Returns (M, k) with k the 1-based global replica index of Eq. 5, or None when no rank exited."""
    if local_key == NO_EXIT:
        key = torch.iinfo(torch.int64).max
    else:
        m, r = local_key >> 32, local_key & 0xFFFFFFFF
        key = (m << 32) | (start + r)
    t = torch.tensor([key], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    g = int(t.item())
    if g == torch.iinfo(torch.int64).max:
        return None
    return g >> 32, (g & 0xFFFFFFFF) + 1


def gelman_rubin_global(means, variances, group=None, device=None):
    """R of Eq. 3 over the replicas of every rank, from this rank's per-replica sample means and
    within-replica variances ([replicas][observables] tensors, FP64): B = mean of squared deviations of
    the replica means, W = mean within-replica variance, R = 1 + B / W (+inf when W <= 0)."""
    means = torch.as_tensor(means, dtype=torch.float64, device=device)
    variances = torch.as_tensor(variances, dtype=torch.float64, device=device)
    sums = torch.stack([means.sum(0), (means * means).sum(0), variances.sum(0),
                        torch.full_like(means[0], float(means.shape[0]))])
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    n = sums[3]
    mean = sums[0] / n
    b = sums[1] / n - mean * mean
    w = sums[2] / n
    return torch.where(w > 0, 1.0 + b / w, torch.full_like(w, float("inf")))


def max_over_ranks(seconds: float, group=None, device=None) -> float:
    """Largest of the ranks' values (tensors on `device`: CUDA for NCCL, CPU for gloo)."""
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
