"""Degenerate batch sizes through the C-ABI on the GPU: a batch of 0 (every
entry point returns without launching and leaves its outputs alone) and a
batch of 1 (one ragged 128-sample tile in every kernel) on the BF16 path of
the 16x16 network (resident grouped sampler, fused backward, strip adjoint)
and on width sets of 144 and 256 spins (grouped sampler with streamed
weights).  Expected values come from the FP64 oracle on the GPU's own
samples."""
import numpy as np
import pytest
import torch

from oracle import made, transfer
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-6  # |delta log Z_R| / N
TOL_RED = 1e-3  # |delta log q| / N in BF16


def _model(graphs, Ws, hidden, betas, seed=5):
    from paper_2504_12037_gb300.model import TNVAN

    return TNVAN(graphs, Ws, hidden, betas, seed=seed, init_scale=1.5)


def _cases():
    w = wl.workload(2)
    yield "16x16", w.graphs[:3], w.widths_sets[:3], w.hidden, w.betas[:3]
    gs = [wl.lattice(24, 24, "gauss", seed=61), wl.lattice(32, 32, "gauss", seed=62)]
    Ws = [wl.width_columns(24, 24, wl.every_kth_column(24)), wl.width_columns(32, 32, wl.every_kth_column(32))]
    yield "streamed", gs, Ws, [128, 128], [0.7, 0.9]


@pytest.mark.parametrize("case", range(2))
def test_batch_zero_leaves_outputs_alone(case):
    name, gs, Ws, hidden, betas = list(_cases())[case]
    model = _model(gs, Ws, hidden, betas)
    spins = torch.full((64,), 5, dtype=torch.int8, device="cuda")
    logq = torch.full((8,), 7.0, dtype=torch.float32, device="cuda")
    logZR = torch.full((8,), 9.0, dtype=torch.float64, device="cuda")
    dbeta = torch.full((8,), 3.0, dtype=torch.float64, device="cuda")
    for prec in (tv.BF16, tv.FP32):
        model.ctx.sample_and_contract(model.betas, 0, 1, 0, prec, spins, logq, logZR)
        model.ctx.sample_contract_adjoint(model.betas, 0, 1, 0, prec, spins, logq, logZR, dbeta)
        model.ctx.contract(model.betas, 0, spins, prec, logZR, dbeta)
        model.ctx.log_prob(0, spins, logq, prec)
    torch.cuda.synchronize()
    assert torch.all(spins == 5) and torch.all(logq == 7.0) and torch.all(logZR == 9.0) and torch.all(dbeta == 3.0)


@pytest.mark.parametrize("case", range(2))
@pytest.mark.parametrize("prec", [tv.BF16, tv.FP32])
def test_batch_of_one(case, prec):
    name, gs, Ws, hidden, betas = list(_cases())[case]
    model = _model(gs, Ws, hidden, betas)
    B = 1
    spins, logq, logZR = model.sample(B, 11, 3, prec)
    torch.cuda.synchronize()
    tol_q = TOL_RED if prec == tv.BF16 else TOL_FP32
    for k, (g, W) in enumerate(zip(gs, Ws)):
        s = torch.as_tensor(model.spins_of(spins, k, B).cpu().numpy().astype(np.float64))
        assert torch.all(s.abs() == 1)
        p = torch.as_tensor(model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy().astype(np.float64))
        lq = made.log_q(p, len(W), hidden, s).numpy()
        assert abs(float(logq[k]) - lq[0]) / g.n <= tol_q, (name, k)
        lz = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, betas[k], W, s, g.Lx).numpy()
        assert abs(float(logZR[k]) - lz[0]) / g.n <= TOL_FP32, (name, k)
    # a training step of one sample per instance: finite outputs, a REINFORCE
    # gradient of zero up to the rounding of the baseline (l_b minus the batch
    # mean is 0), statistics of n = 1
    out = model.buffers(B)
    dbeta = torch.empty(model.n * B, dtype=torch.float64, device="cuda")
    model.train_step(B, 13, 0, prec, 0.01, out, dbeta, None)
    torch.cuda.synchronize()
    assert torch.isfinite(out[1]).all() and torch.isfinite(out[2]).all() and torch.isfinite(dbeta).all()
    assert torch.isfinite(model.params).all()
    assert float(model.grad.abs().max()) <= 1e-6
    st = model.step_stats().cpu().numpy()
    assert np.all(st[:, 7] == 1) and np.all(st[:, 5] == 0) and np.all(st[:, 6] == 0)
