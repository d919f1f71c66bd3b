"""GPU parity of tnvan_observables (importance-weighted internal energy and
bond correlations from one batch; strip, dense and elimination instances)
against the FP64 oracle, through the C-ABI.  Samples and log q are seeded
inputs; the oracle contracts every sample exactly and differentiates it with
autograd."""
import numpy as np
import pytest
import torch

from oracle import estimators as est
from oracle import general, transfer
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import to_dev_spins

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [0, 1, 32, 128])
def test_observables_match_oracle(shape):
    # strips of width 1-4, 20 rows, a ragged batch of 40 rows
    Lx, Ly, beta, batch = 14, 20, 0.7, 40
    g = wl.lattice(Lx, Ly, "gauss", seed=93)
    W = wl.width_columns(Lx, Ly, [1, 4, 8, 13])
    from paper_2504_12037_gb300.model import TNVAN

    model = TNVAN([g], [W], [32, 32], [beta], seed=5)
    model.ctx.set_tuning((0, 0, 0, shape, 0, 0))
    D = len(W)
    rng = np.random.default_rng(23)
    s = np.where(rng.random((batch, D)) < 0.5, 1.0, -1.0)
    lq = rng.normal(-D * np.log(2.0), 3.0, size=batch).astype(np.float32)
    # oracle: exact log Z_R per sample, self-normalised weights, d/dbeta and
    # the weighted d/dJ by autograd
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lz = transfer.log_zr_lattice(g.n, g.ei, g.ej, Jt, bt, W, torch.as_tensor(s), g.Lx)
    l = lz.detach() - torch.as_tensor(lq, dtype=torch.float64)
    wts = torch.softmax(l, 0)
    db = torch.stack([torch.autograd.grad(lz[b], bt, retain_graph=True)[0] for b in range(batch)])
    (corr_ref,) = torch.autograd.grad((wts * lz).sum(), Jt)
    U_ref, Uq_ref, ess_ref = est.is_observables(lz.detach(), torch.as_tensor(lq, dtype=torch.float64), -db)
    # GPU
    d_spins = to_dev_spins(s.reshape(-1))
    logZR = torch.empty(batch, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR)
    logq = torch.as_tensor(lq).cuda()
    corr = torch.full((g.m,), float("nan"), dtype=torch.float64, device="cuda")
    out = model.ctx.observables(model.betas, batch, d_spins, logZR, logq, corr)
    torch.cuda.synchronize()
    U, Uq, ess = out[0]
    assert abs(U - U_ref) <= 2e-5 * abs(U_ref)
    assert abs(Uq - Uq_ref) <= 2e-5 * abs(Uq_ref)
    assert abs(ess - ess_ref) <= 1e-4 * ess_ref
    assert 1.0 <= ess <= batch
    assert float((corr.cpu() - corr_ref).abs().max()) <= 2e-5 * max(1.0, float(corr_ref.abs().max()))
    # energies alone are the same numbers
    out2 = model.ctx.observables(model.betas, batch, d_spins, logZR, logq)
    torch.cuda.synchronize()
    assert np.array_equal(out, out2)


def test_observables_uniform_weights_reduce_to_batch_means():
    # equal l_b (log q = log Z_R) make every weight 1/B: U = U_q, ESS = B, and
    # the weighted d/dJ equals tnvan_backward's batch-mean d/dJ
    w = wl.workload(2)
    from paper_2504_12037_gb300.model import TNVAN

    model = TNVAN(w.graphs[:2], w.widths_sets[:2], w.hidden, w.betas[:2], seed=8)
    B = 500
    spins, logq, logZR = model.sample(B, 4, 2, tv.FP32)
    lq_eq = logZR.float()  # l_b = 0 up to the FP32 rounding of log q
    corr = torch.empty(sum(model.n_edges), dtype=torch.float64, device="cuda")
    out = model.ctx.observables(model.betas, B, spins, logZR, lq_eq, corr)
    grad = torch.empty_like(model.params)
    dJ = torch.empty_like(corr)
    model.ctx.backward(model.betas, B, spins, logZR, lq_eq, tv.FP32, grad, None, dJ)
    torch.cuda.synchronize()
    for k in range(2):
        U, Uq, ess = out[k]
        assert abs(U - Uq) <= 1e-3 * abs(Uq)
        assert abs(ess - B) <= 1e-2 * B
    assert float((corr - dJ).abs().max()) <= 1e-3 * float(dJ.abs().max())


def test_observables_dense_instance_match_oracle():
    # SK block: the dense adjoint's weighted pair and single-spin marginals
    # and the weighted W-W bond sums
    from oracle import dense
    from paper_2504_12037_gb300.model import TNVAN

    g = wl.sk(18, 4)
    W = np.arange(6, 18, dtype=np.int32)
    beta, batch = 1.1, 37
    model = TNVAN([g], [W], [16], [beta], seed=2)
    D = len(W)
    rng = np.random.default_rng(31)
    s = np.where(rng.random((batch, D)) < 0.5, 1.0, -1.0)
    lq = rng.normal(-D * np.log(2.0), 2.0, size=batch).astype(np.float32)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lz = dense.log_zr_dense(g.n, g.ei, g.ej, Jt, bt, W, torch.as_tensor(s))
    l = lz.detach() - torch.as_tensor(lq, dtype=torch.float64)
    wts = torch.softmax(l, 0)
    db = torch.stack([torch.autograd.grad(lz[b], bt, retain_graph=True)[0] for b in range(batch)])
    (corr_ref,) = torch.autograd.grad((wts * lz).sum(), Jt)
    U_ref, Uq_ref, ess_ref = est.is_observables(lz.detach(), torch.as_tensor(lq, dtype=torch.float64), -db)
    d_spins = to_dev_spins(s.reshape(-1))
    logZR = torch.empty(batch, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR)
    logq = torch.as_tensor(lq).cuda()
    corr = torch.full((g.m,), float("nan"), dtype=torch.float64, device="cuda")
    out = model.ctx.observables(model.betas, batch, d_spins, logZR, logq, corr)
    torch.cuda.synchronize()
    U, Uq, ess = out[0]
    assert abs(U - U_ref) <= 2e-5 * abs(U_ref)
    assert abs(Uq - Uq_ref) <= 2e-5 * abs(Uq_ref)
    assert abs(ess - ess_ref) <= 1e-4 * ess_ref
    assert float((corr.cpu() - corr_ref).abs().max()) <= 2e-5 * max(1.0, float(corr_ref.abs().max()))


@pytest.mark.parametrize("wu", [2, 6])
def test_observables_elimination_instance_match_oracle(wu):
    # a random regular graph with a finder-planned width set: the weighted
    # bond sums of the elimination reverse sweep and of the W-W bonds
    g = wl.random_regular(120, 3, 12037 + 8100 + wu)
    W, order, _, _ = tv.find_width_set(g.n, g.ei, g.ej, wu, restarts=2, seed=3)
    beta, batch = 0.8, 52
    from paper_2504_12037_gb300.model import TNVAN

    model = TNVAN([g], [W], [16], [beta], seed=5, elim_orders=[order])
    D = len(W)
    rng = np.random.default_rng(29)
    s = np.where(rng.random((batch, D)) < 0.5, 1.0, -1.0)
    lq = rng.normal(-D * np.log(2.0), 3.0, size=batch).astype(np.float32)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lz = general.log_zr_general(g.n, g.ei, g.ej, Jt, bt, W, torch.as_tensor(s))
    l = lz.detach() - torch.as_tensor(lq, dtype=torch.float64)
    wts = torch.softmax(l, 0)
    db = torch.stack([torch.autograd.grad(lz[b], bt, retain_graph=True)[0] for b in range(batch)])
    (corr_ref,) = torch.autograd.grad((wts * lz).sum(), Jt)
    U_ref, Uq_ref, ess_ref = est.is_observables(lz.detach(), torch.as_tensor(lq, dtype=torch.float64), -db)
    d_spins = to_dev_spins(s.reshape(-1))
    logZR = torch.empty(batch, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR)
    logq = torch.as_tensor(lq).cuda()
    corr = torch.full((g.m,), float("nan"), dtype=torch.float64, device="cuda")
    out = model.ctx.observables(model.betas, batch, d_spins, logZR, logq, corr)
    torch.cuda.synchronize()
    U, Uq, ess = out[0]
    assert abs(U - U_ref) <= 2e-5 * abs(U_ref)
    assert abs(Uq - Uq_ref) <= 2e-5 * abs(Uq_ref)
    assert abs(ess - ess_ref) <= 1e-4 * ess_ref
    assert float((corr.cpu() - corr_ref).abs().max()) <= 2e-5 * max(1.0, float(corr_ref.abs().max()))
