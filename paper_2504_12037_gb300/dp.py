"""Data-parallel exchange for training one network across ranks.

Samples are independent (Eq. 9-10 are batch means), so a data-parallel step
needs exactly one exchange: the per-rank reduction statistics and the
per-rank gradient.  The statistics travel as the associative FP64 tuple
  (n, sum l, sum l^2, logsumexp l)
from which F_q, its standard error and the importance-sampled log Z of the
union of all ranks' samples follow; tuples are all-gathered and merged in
rank order, so every rank gets the same, deterministic result.  Gradients are
averaged with one all-reduce (each rank's REINFORCE weights use its own batch
mean as baseline, which keeps the estimator unbiased).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np
import torch
import torch.distributed as dist


def tuple_from_stats(fe_row: Sequence[float], n: int, beta: float) -> np.ndarray:
    """Rebuild (n, sum l, sum l^2, logsumexp l) from one instance's
    tnvan_free_energy output [F_q, F_IS, stderr, logZ_IS] over n samples."""
    F_q, _, se, lz = (float(x) for x in fe_row[:4])
    mean = -beta * F_q
    var = (se * beta) ** 2 * n
    s1 = n * mean
    s2 = (n - 1) * var + n * mean * mean
    return np.array([n, s1, s2, lz + math.log(n)], dtype=np.float64)


def merge_tuples(tuples: Sequence[np.ndarray]) -> np.ndarray:
    n = sum(t[0] for t in tuples)
    s1 = sum(t[1] for t in tuples)
    s2 = sum(t[2] for t in tuples)
    m = max(t[3] for t in tuples)
    lse = m + math.log(sum(math.exp(t[3] - m) for t in tuples))
    return np.array([n, s1, s2, lse], dtype=np.float64)


def stats_from_tuple(t: np.ndarray, beta: float) -> dict:
    n, s1, s2, lse = (float(x) for x in t)
    mean = s1 / n
    var = max(s2 - s1 * mean, 0.0) / (n - 1) if n > 1 else 0.0
    lz = lse - math.log(n)
    return {"F_q": -mean / beta, "F_IS": -lz / beta, "stderr": math.sqrt(var / n) / beta, "logZ_IS": lz}


def allreduce_free_energy(fe: np.ndarray, n_local: int, betas: Sequence[float], group=None) -> np.ndarray:
    """fe: this rank's [n_inst, 4] tnvan_free_energy output.  Returns the
    [n_inst, 4] statistics of all ranks' samples together (same on every rank)."""
    world = dist.get_world_size(group)
    local = np.stack([tuple_from_stats(fe[k], n_local, betas[k]) for k in range(len(betas))])
    buf = [torch.zeros(local.shape, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(buf, torch.as_tensor(local), group=group)
    out = np.zeros((len(betas), 4))
    for k in range(len(betas)):
        st = stats_from_tuple(merge_tuples([b.numpy()[k] for b in buf]), betas[k])
        out[k] = [st["F_q"], st["F_IS"], st["stderr"], st["logZ_IS"]]
    return out


def allreduce_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Average the flat gradient over ranks (in place)."""
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    grad /= dist.get_world_size(group)
    return grad
