"""Multi-GPU runs as independent replicas (one process per GPU).

Ensemble members are independent (no exchange while stepping), so N GPUs run N
replicas: rank r steps its own ensemble whose members draw from disjoint counter ranges
of the SplitMix64 stream (weak scaling, no collective on the data path).  After the
run, the host gathers per-member results and timings; the ensemble statistics of
Sec. 3.3 Eq. (41) (mean over members, here with its standard error) are computed over
all ranks' members.  The functions take a torch.distributed process group (NCCL on
GPUs, gloo on CPU).
"""
import math

import numpy as np


def member_counter_base(rank, members_per_rank, points_per_member):
    """First SplitMix64 draw index of rank `rank`'s member 0 (ranks use disjoint ranges)."""
    return rank * members_per_rank * points_per_member


def member_range(rank, world, m):
    """Contiguous, balanced share [lo, hi) of m members for rank `rank` (for sharding one
    ensemble across ranks instead of replicating it)."""
    base, extra = divmod(m, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest value of x over the ranks of the default group (x itself if not distributed)."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_members(values, dist=None, device="cpu"):
    """Concatenate every rank's per-member array (equal shapes) along the member axis
    (axis 0), rank order: per-member scalars, or per-member sample series (members x T)
    whose ensemble moments are then taken over all ranks' members."""
    values = np.asarray(values, dtype=np.float64)
    if dist is None or not dist.is_initialized():
        return values
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return np.concatenate([o.cpu().numpy() for o in out])


def ensemble_stats(values, labels):
    """Mean, standard error (s / sqrt(n)) and count of `values` per distinct label, e.g. the
    time-averaged beta of every member grouped by its initial mean C0.  Non-finite values
    (runs that never reached the averaging window) are left out."""
    values = np.asarray(values, dtype=np.float64)
    labels = np.asarray(labels)
    out = {}
    for lab in sorted(set(labels.tolist())):
        v = values[(labels == lab) & np.isfinite(values)]
        n = v.size
        mean = float(v.mean()) if n else float("nan")
        se = float(v.std(ddof=1) / math.sqrt(n)) if n > 1 else float("nan")
        out[lab] = {"mean": mean, "se": se, "n": int(n)}
    return out
