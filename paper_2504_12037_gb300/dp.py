"""Data-parallel training of one set of networks across ranks.

Samples are independent (Eq. 9-10 are batch means), so one training step of
a batch split over ranks needs two small exchanges around the local work:

  1. every rank samples and contracts its share (own Philox stream) and
     reduces it to Eq. 9 statistics rows (tnvan_reduce: F_q, F_IS, stderr,
     logZ_IS, mean l, #non-finite, var l, n per instance);
  2. the rows are all-gathered and merged in rank order into the rows of the
     union batch (tnvan_merge_stats on the device; `merge_stats` below is the
     same merge on the host) -- counts add, means and second central moments
     combine by the pairwise update of Chan, Golub and LeVeque (1979), and the
     importance weights' log-sums by logaddexp -- so every rank holds the
     same global baseline and batch size;
  3. each rank's REINFORCE gradient uses that global baseline and batch size
     (tnvan_backward_stats), so one all-reduce (sum) of the gradients gives
     exactly the gradient of the union batch (Eq. 10), and every rank takes
     the same Adam step.

The payload per step is 8 doubles per instance per rank plus one gradient.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import torch
import torch.distributed as dist

# statistics row layout (tnvan_reduce / tnvan_step_stats / tnvan_merge_stats)
F_Q, F_IS, STDERR, LOGZ_IS, MEAN, BAD, VAR, N = range(8)


def merge_stats(parts: np.ndarray, betas) -> np.ndarray:
    """Host form of tnvan_merge_stats: parts [n_parts, n_inst, 8] -> [n_inst, 8]
    for the union of the parts (parts merged in index order, FP64)."""
    parts = np.asarray(parts, np.float64)
    if parts.shape[0] == 1:
        return parts[0].copy()
    out = np.zeros(parts.shape[1:], np.float64)
    for k in range(parts.shape[1]):
        n = mean = M2 = lse = bad = 0.0
        for p in range(parts.shape[0]):
            q = parts[p, k]
            bad += q[BAD]
            nb = q[N]
            if not nb > 0:
                continue
            mb, M2b, lb = q[MEAN], q[VAR] * (nb - 1) if nb > 1 else 0.0, q[LOGZ_IS] + math.log(nb)
            if n == 0:
                n, mean, M2, lse = nb, mb, M2b, lb
                continue
            tot = n + nb
            d = mb - mean
            mean += d * (nb / tot)
            M2 += M2b + d * d * (n * nb / tot)
            lse = max(lse, lb) + math.log1p(math.exp(-abs(lse - lb)))
            n = tot
        beta = float(betas[k])
        var = M2 / (n - 1) if n > 1 else 0.0
        lz = lse - math.log(n) if n > 0 else float("nan")
        out[k] = [-mean / beta, -lz / beta, math.sqrt(var) / (beta * math.sqrt(n)) if n > 0 else float("nan"),
                  lz, mean, bad, var, n]
    return out


def gather_stats(local: torch.Tensor, group=None) -> torch.Tensor:
    """All-gather every rank's statistics rows [n_inst, 8] -> [world, n_inst, 8]
    (rank order), on the device of `local`."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        return local.reshape(1, *local.shape).clone()
    bufs = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(bufs, local.contiguous(), group=group)
    return torch.stack(bufs)


def sum_gradient(grad: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the per-rank gradients in place (each already carries 1/B_total)."""
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad


class DataParallelStep:
    """One data-parallel training step of a TNVAN model (every rank holds the
    same networks): local sampling with the contraction adjoint, the
    statistics exchange, the local gradient with the global baseline, the
    gradient all-reduce and Adam.  `batch` is this rank's share per instance;
    the rank's Philox stream is its own (seed offset by the rank)."""

    def __init__(self, model, batch: int, precision: int, lr: float = 0.01, group=None,
                 dbeta: Optional[torch.Tensor] = None, dJ: Optional[torch.Tensor] = None):
        self.model, self.batch, self.precision, self.lr, self.group = model, batch, precision, lr, group
        self.out = model.buffers(batch)
        self.dbeta, self.dJ = dbeta, dJ
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.local = torch.empty(model.n, 8, dtype=torch.float64, device=model.device)
        self.merged = torch.empty(model.n, 8, dtype=torch.float64, device=model.device)

    def __call__(self, seed: int, step: int, stream=None):
        m, B = self.model, self.batch
        spins, logq, logZR = self.out
        m.ctx.sample_contract_adjoint(m.betas, B, seed + 7919 * self.rank, step, self.precision, spins, logq, logZR,
                                      self.dbeta, self.dJ, stream)
        m.ctx.reduce(m.betas, B, logZR, logq, self.local, stream)
        parts = gather_stats(self.local, self.group)
        m.ctx.merge_stats(m.betas, parts, self.merged, stream)
        m.ctx.backward_stats(m.betas, B, spins, logZR, logq, self.precision, m.grad, stream)
        sum_gradient(m.grad, self.group)
        m.t += 1
        m.ctx.adam(m.params, m.grad, m.m, m.v, self.lr, 0.9, 0.999, 1e-8, m.t, stream)
        return self.merged
