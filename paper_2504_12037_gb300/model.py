"""Multi-instance TNVAN driver over the C-ABI (Algorithm 1).

`TNVAN` registers every (graph, width set, beta) instance in one library
context, owns the flat float32 parameter vector of all instances' networks,
and runs Algorithm 1's loop: (a) sample, (b) contract, (c) F_q and its
gradient, (d) Adam update -- each a call into libtnvan's kernels.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np
import torch

from . import tnvan as tv
from .workloads import Graph, made_param_count, made_params


class TNVAN:
    def __init__(self, graphs: Sequence[Graph], width_sets: Sequence[np.ndarray], hidden: Sequence[int],
                 betas: Sequence[float], device: int = 0, seed: int = 0, init_scale: float = 1.0,
                 params: Optional[np.ndarray] = None, elim_orders: Optional[Sequence] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("TNVAN needs a CUDA device")
        self.device = torch.device("cuda", device)
        self.ctx = tv.Context(device)
        self.n = len(graphs)
        self.betas = np.asarray(betas, np.float64)
        self.hidden = list(hidden)
        self.D = [int(len(W)) for W in width_sets]
        self.graphs = list(graphs)
        for k, (g, W) in enumerate(zip(graphs, width_sets)):
            self.ctx.init_graph(k, g.n, g.ei, g.ej, g.J, g.topology, g.Lx, g.Ly, g.periodic)
            self.ctx.set_width_set(k, W, None if elim_orders is None else elim_orders[k])
        sizes = [made_param_count(D, hidden) for D in self.D]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        if params is None:
            params = np.concatenate([made_params(D, hidden, seed + k, init_scale) for k, D in enumerate(self.D)])
        self.params = torch.as_tensor(np.asarray(params, np.float32)).to(self.device)
        for k in range(self.n):
            self.ctx.set_made(k, self.hidden, self.params[self.offsets[k]:self.offsets[k + 1]])
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.n_edges = [g.m for g in graphs]

    def buffers(self, batch: int):
        spins = torch.empty(batch * sum(self.D), dtype=torch.int8, device=self.device)
        logq = torch.empty(self.n * batch, dtype=torch.float32, device=self.device)
        logZR = torch.empty(self.n * batch, dtype=torch.float64, device=self.device)
        return spins, logq, logZR

    def spins_of(self, spins: torch.Tensor, k: int, batch: int) -> torch.Tensor:
        off = batch * sum(self.D[:k])
        return spins[off:off + batch * self.D[k]].view(batch, self.D[k])

    def sample(self, batch: int, seed: int, step: int, precision: int = tv.FP32, out=None, stream=None):
        spins, logq, logZR = out if out is not None else self.buffers(batch)
        self.ctx.sample_and_contract(self.betas, batch, seed, step, precision, spins, logq, logZR, stream)
        return spins, logq, logZR

    def capture_train_step(self, batch: int, seed: int, precision: int = tv.FP32, lr: float = 0.01, out=None,
                           dbeta=None, dJ=None) -> "CapturedStep":
        """The training step as a replayable CUDA graph (see CapturedStep)."""
        return CapturedStep(self, batch, seed, precision, lr, out, dbeta, dJ)

    def free_energy(self, batch: int, logZR, logq, stream=None) -> np.ndarray:
        """[n_inst, 4]: F_q, F_IS, stderr, logZ_IS (per instance, not per spin)."""
        return self.ctx.free_energy(self.betas, batch, logZR, logq, stream)

    def step_stats(self, out=None, stream=None) -> torch.Tensor:
        """Device [n_inst, 8] Eq. 9 rows of the last training step (F_q, F_IS,
        stderr, logZ_IS, mean l, #non-finite, var l, n), queued on `stream`."""
        out = torch.empty(8 * self.n, dtype=torch.float64, device=self.device) if out is None else out
        self.ctx.step_stats(out, stream)
        return out.view(self.n, 8)

    def train_step(self, batch: int, seed: int, step: int, precision: int = tv.FP32, lr: float = 0.01,
                   out=None, dbeta=None, dJ=None, stream=None):
        """One iteration of Algorithm 1: sample, contract, gradient, Adam, in one
        library call (tnvan_train_step).  With dbeta / dJ given, the
        contraction adjoint runs in the sampling pass."""
        spins, logq, logZR = out if out is not None else self.buffers(batch)
        self.t += 1
        self.ctx.train_step(self.betas, batch, seed, step, precision, spins, logq, logZR, dbeta, dJ, self.grad,
                            self.m, self.v, lr, 0.9, 0.999, 1e-8, self.t, stream)
        return spins, logq, logZR

    def train_step_separate(self, batch: int, seed: int, step: int, precision: int = tv.FP32, lr: float = 0.01,
                            out=None, dbeta=None, dJ=None, stream=None):
        """train_step through the separate entry points (sampling with the
        adjoint, backward, Adam): the same step, three calls."""
        spins, logq, logZR = out if out is not None else self.buffers(batch)
        self.ctx.sample_contract_adjoint(self.betas, batch, seed, step, precision, spins, logq, logZR, dbeta, dJ,
                                         stream)
        self.ctx.backward(self.betas, batch, spins, logZR, logq, precision, self.grad, None, None, stream)
        self.t += 1
        self.ctx.adam(self.params, self.grad, self.m, self.v, lr, 0.9, 0.999, 1e-8, self.t, stream)
        return spins, logq, logZR


class CapturedStep:
    """One training step (Algorithm 1 (a)-(d): sample, contract with the
    adjoint, REINFORCE gradient, Adam) captured once as a CUDA graph.

    Each replay() runs the whole step on the device with no host work: the
    Philox step of the sampler and Adam's t advance through a device counter
    (tnvan_set_step_counter), so every replay draws fresh samples into the
    same buffers (`out`, `dbeta`, `dJ`) and leaves the step's Eq. 9 rows
    (F_q, F_IS, stderr, logZ_IS, ...) in `stats` [n_inst, 8].  Construction
    takes one eager step (workspaces and launch plans settle) before
    capturing."""

    def __init__(self, model: "TNVAN", batch: int, seed: int, precision: int = tv.FP32, lr: float = 0.01,
                 out=None, dbeta=None, dJ=None):
        self.model = model
        self.out = out if out is not None else model.buffers(batch)
        self.dbeta, self.dJ = dbeta, dJ
        self.counter = torch.zeros(1, dtype=torch.int64, device=model.device)
        self.stats = torch.zeros(model.n, 8, dtype=torch.float64, device=model.device)
        self.stream = torch.cuda.Stream(device=model.device)
        self.stream.wait_stream(torch.cuda.current_stream(model.device))
        model.ctx.reserve(batch)
        with torch.cuda.stream(self.stream):
            model.train_step(batch, seed, 0, precision, lr, self.out, dbeta, dJ, self.stream)
        self.stream.synchronize()
        model.ctx.set_step_counter(self.counter)
        self.graph = torch.cuda.CUDAGraph()
        t0 = model.t
        with torch.cuda.graph(self.graph, stream=self.stream):
            model.train_step(batch, seed, 1, precision, lr, self.out, dbeta, dJ, self.stream)
            model.ctx.step_stats(self.stats, self.stream)
            self.counter.add_(1)
        model.t = t0  # the graph's step is t0 + 1 + counter
        model.ctx.set_step_counter(None)

    def replay(self):
        """One training step, queued on the current stream."""
        self.graph.replay()
        self.model.t += 1


class FreeEnergyFunction(torch.autograd.Function):
    """F_q of every instance as a differentiable function of the network
    parameters and the couplings J (Eq. 9 forward, Eq. 10 and the contraction
    adjoint backward).  The forward draws a fresh batch."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, J: torch.Tensor, model: TNVAN, batch: int, seed: int, step: int,
                precision: int = tv.FP32):
        spins, logq, logZR = model.sample(batch, seed, step, precision)
        fe = model.free_energy(batch, logZR, logq)
        ctx.model, ctx.batch, ctx.precision = model, batch, precision
        ctx.save_for_backward(spins, logq, logZR)
        return torch.as_tensor(fe[:, 0], dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, g_out: torch.Tensor):
        spins, logq, logZR = ctx.saved_tensors
        model = ctx.model
        grad = torch.empty_like(model.params)
        dJ = torch.empty(sum(model.n_edges), dtype=torch.float64, device=grad.device)
        model.ctx.backward(model.betas, ctx.batch, spins, logZR, logq, ctx.precision, grad, None, dJ)
        scale_p = torch.repeat_interleave(g_out.float(), torch.as_tensor(np.diff(model.offsets), device=grad.device))
        eoff = torch.as_tensor(model.n_edges, device=grad.device)
        beta = torch.as_tensor(model.betas, device=grad.device)
        # F_q = -(1/beta) mean(log Z_R - log q) and q does not depend on J
        scale_j = torch.repeat_interleave(-g_out / beta, eoff)
        return grad * scale_p, dJ * scale_j, None, None, None, None, None
