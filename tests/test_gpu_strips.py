"""GPU parity of the lattice-strip path (4x4 +-J and 16x16 Gaussian
workloads) against the FP64 oracle, through the C-ABI."""
import math

import numpy as np
import pytest
import torch

from oracle import estimators as est
from oracle import ising, made, transfer
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import check_sample_agreement, oracle_samples, to_dev_spins

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-6  # |delta log Z| / N and |delta log q| / N


def _model(w, n_inst=None, seed=3, scale=1.0):
    from paper_2504_12037_gb300.model import TNVAN

    n = len(w.graphs) if n_inst is None else n_inst
    return TNVAN(w.graphs[:n], w.widths_sets[:n], w.hidden, w.betas[:n], seed=seed, init_scale=scale)


def _param_mask(D, hidden):
    """1 where a parameter is inside the MADE masks (biases always), flat layout."""
    parts = []
    for m in made.masks(D, hidden):
        parts.append(m.numpy().reshape(-1))
        parts.append(np.ones(m.shape[0]))
    return np.concatenate(parts)


def _oracle_logzr(g, W, s, beta):
    if g.n <= 16:
        return ising.log_zr_enum(g.n, g.ei, g.ej, g.J, beta, W, s)
    return transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, beta, W, s, g.Lx)


@pytest.mark.parametrize("cfg,batch", [(1, 1024), (2, 192)])
def test_sampler_replay_logq_logzr(cfg, batch):
    w = wl.workload(cfg)
    model = _model(w, scale=2.0)
    seed, step = 12037, 4
    spins, logq, logZR = model.sample(batch, seed, step)
    torch.cuda.synchronize()
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, p_or, u = oracle_samples(p32, D, w.hidden, seed, step, k, batch)
        s_gpu = model.spins_of(spins, k, batch).cpu().numpy().astype(np.float64)
        same = check_sample_agreement(s_gpu, s_or.numpy(), u, p_or.numpy())
        lq_or = made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, w.hidden, s_or)
        lz_or = _oracle_logzr(g, W, s_or, beta)
        lq_gpu = logq[k * batch:(k + 1) * batch].cpu().double()
        lz_gpu = logZR[k * batch:(k + 1) * batch].cpu()
        m = torch.as_tensor(same)
        assert float((lq_gpu[m] - lq_or[m]).abs().max()) / g.n <= TOL_FP32
        assert float((lz_gpu[m] - lz_or[m]).abs().max()) / g.n <= TOL_FP32


@pytest.mark.parametrize("cfg,batch", [(1, 333), (2, 97)])
def test_contract_and_log_prob_on_oracle_samples(cfg, batch):
    w = wl.workload(cfg)
    model = _model(w, scale=1.5)
    s_all, lq_all, lz_all = [], [], []
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, D, w.hidden, 99, 0, k, batch)
        s_all.append(s_or.numpy().reshape(-1))
        lq_all.append(made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, w.hidden, s_or))
        lz_all.append(_oracle_logzr(g, W, s_or, beta))
    d_spins = to_dev_spins(np.concatenate(s_all))
    logq = torch.empty(model.n * batch, dtype=torch.float32, device="cuda")
    logZR = torch.empty(model.n * batch, dtype=torch.float64, device="cuda")
    model.ctx.log_prob(batch, d_spins, logq)
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR)
    torch.cuda.synchronize()
    for k in range(model.n):
        n = w.graphs[k].n
        assert float((logq[k * batch:(k + 1) * batch].cpu().double() - lq_all[k]).abs().max()) / n <= TOL_FP32
        assert float((logZR[k * batch:(k + 1) * batch].cpu() - lz_all[k]).abs().max()) / n <= TOL_FP32


def test_contract_edge_configurations():
    # all up, all down, alternating and a single flipped spin on the 16x16 lattice
    w = wl.workload(2)
    model = _model(w, n_inst=2)
    D = model.D[0]
    rows = [np.ones(D), -np.ones(D), np.array([(-1) ** i for i in range(D)], float)]
    r = np.ones(D)
    r[17] = -1
    rows.append(r)
    s = np.stack(rows)
    B = s.shape[0]
    d_spins = to_dev_spins(np.concatenate([s.reshape(-1)] * 2))
    logZR = torch.empty(2 * B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, logZR)
    torch.cuda.synchronize()
    for k in range(2):
        g, W = w.graphs[k], w.widths_sets[k]
        ref = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, w.betas[k], W, torch.as_tensor(s), g.Lx)
        assert float((logZR[k * B:(k + 1) * B].cpu() - ref).abs().max()) / g.n <= TOL_FP32


def test_free_energy_reduction_matches_oracle():
    w = wl.workload(2)
    model = _model(w)
    B = 5000
    rng = np.random.default_rng(1)
    lz = rng.normal(-300, 3, size=(model.n, B))
    lq = rng.normal(-40, 2, size=(model.n, B)).astype(np.float32)
    out = model.ctx.free_energy(model.betas, B, torch.as_tensor(lz.reshape(-1)).cuda(),
                                torch.as_tensor(lq.reshape(-1)).cuda())
    for k in range(model.n):
        ref = est.free_energies(lz[k], lq[k].astype(np.float64), model.betas[k])
        N = w.graphs[k].n
        assert abs(out[k, 0] - ref["F_q"]) / N < 1e-9
        assert abs(out[k, 1] - ref["F_IS"]) / N < 1e-7
        assert abs(out[k, 3] - ref["logZ_IS"]) / N < 1e-7
        assert abs(out[k, 2] - ref["stderr"]) < 1e-6 * ref["stderr"]
        assert out[k, 1] <= out[k, 0]


def test_free_energy_single_sample_and_nonfinite():
    w = wl.workload(1)
    model = _model(w)
    out = model.ctx.free_energy(model.betas, 1, torch.tensor([-3.5], dtype=torch.float64, device="cuda"),
                                torch.tensor([-1.25], dtype=torch.float32, device="cuda"))
    assert abs(out[0, 0] - 2.25) < 1e-12 and abs(out[0, 1] - 2.25) < 1e-7
    with pytest.raises(tv.TnvanError) as e:
        model.ctx.free_energy(model.betas, 2, torch.tensor([float("nan"), 1.0], dtype=torch.float64, device="cuda"),
                              torch.zeros(2, dtype=torch.float32, device="cuda"))
    assert e.value.code == tv.E_OVERFLOW


@pytest.mark.parametrize("cfg,batch", [(1, 300), (2, 70)])
def test_reinforce_gradient_matches_oracle(cfg, batch):
    w = wl.workload(cfg)
    model = _model(w, scale=1.5)
    s_all, lq_all, lz_all, ref = [], [], [], []
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        th = torch.as_tensor(p32, dtype=torch.float64)
        s_or, _, _ = oracle_samples(p32, D, w.hidden, 7, 1, k, batch)
        lq = made.log_q(th, D, w.hidden, s_or).float().double()  # as the GPU stores it
        lz = _oracle_logzr(g, W, s_or, beta)
        wts = est.reinforce_weights(lz, lq, beta)
        ref.append(est.surrogate_grad(p32.astype(np.float64), D, w.hidden, s_or, wts))
        s_all.append(s_or.numpy().reshape(-1))
        lq_all.append(lq.numpy())
        lz_all.append(lz.detach().numpy())
    d_spins = to_dev_spins(np.concatenate(s_all))
    logq = torch.as_tensor(np.concatenate(lq_all), dtype=torch.float32).cuda()
    logZR = torch.as_tensor(np.concatenate(lz_all)).cuda()
    grad = torch.full_like(model.params, float("nan"))
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, tv.FP32, grad)
    torch.cuda.synchronize()
    for k in range(model.n):
        gk = grad[model.offsets[k]:model.offsets[k + 1]].cpu().double()
        scale = float(ref[k].abs().max())
        assert float((gk - ref[k]).abs().max()) <= 2e-5 * scale + 1e-9


@pytest.mark.parametrize("cfg,batch", [(1, 64), (2, 24)])
def test_contraction_adjoint_beta_and_J(cfg, batch):
    w = wl.workload(cfg)
    model = _model(w)
    n_inst = model.n
    s_all, db_ref, dj_ref = [], [], []
    for k in range(n_inst):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, D, w.hidden, 5, 2, k, batch)
        bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
        lz = transfer.log_zr_lattice(g.n, g.ei, g.ej, Jt, bt, W, s_or, g.Lx)
        db = torch.stack([torch.autograd.grad(lz[b], bt, retain_graph=True)[0] for b in range(batch)])
        (dj,) = torch.autograd.grad(lz.mean(), Jt)
        db_ref.append(db)
        dj_ref.append(dj)
        s_all.append(s_or.numpy().reshape(-1))
    d_spins = to_dev_spins(np.concatenate(s_all))
    dbeta = torch.empty(n_inst * batch, dtype=torch.float64, device="cuda")
    logZR = torch.empty(n_inst * batch, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR, dbeta)
    logq = torch.zeros(n_inst * batch, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(model.params)
    dJ = torch.empty(sum(model.n_edges), dtype=torch.float64, device="cuda")
    db2 = torch.empty_like(dbeta)
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, tv.FP32, grad, db2, dJ)
    torch.cuda.synchronize()
    eo = 0
    for k in range(n_inst):
        N = w.graphs[k].n
        ref = db_ref[k]
        got = dbeta[k * batch:(k + 1) * batch].cpu()
        assert float((got - ref).abs().max()) <= 2e-5 * float(ref.abs().max())
        # the backward pass forms d/dbeta from the bond expectations of its
        # reverse sweep (sum_e J_e <s s>_e - E_1), not by forward mode
        got2 = db2[k * batch:(k + 1) * batch].cpu()
        assert float((got2 - ref).abs().max()) <= 2e-5 * float(ref.abs().max())
        m = w.graphs[k].m
        gj = dJ[eo:eo + m].cpu()
        assert float((gj - dj_ref[k]).abs().max()) <= 2e-5 * max(1.0, float(dj_ref[k].abs().max()))
        eo += m


@pytest.mark.parametrize("shape", [0, 1, 32, 128])
def test_strip_adjoint_all_widths_tall_strips(shape):
    # strips of width 1, 2, 3 and 4 and 20 rows (more than one 16-row pass),
    # a ragged batch of 40 seeded spin rows: d/dbeta per sample and the
    # batch-mean d/dJ against FP64 autograd through the oracle's contraction;
    # every launch shape of the adjoint (0 = default, 1 = one warp per strip,
    # else samples per CTA)
    Lx, Ly, beta, batch = 14, 20, 0.7, 40
    g = wl.lattice(Lx, Ly, "gauss", seed=91)
    W = wl.width_columns(Lx, Ly, [1, 4, 8, 13])
    from paper_2504_12037_gb300.model import TNVAN

    model = TNVAN([g], [W], [32, 32], [beta], seed=5)
    model.ctx.set_tuning((0, 0, 0, shape, 0, 0))
    D = len(W)
    s = np.where(np.random.default_rng(17).random((batch, D)) < 0.5, 1.0, -1.0)
    s_t = torch.as_tensor(s)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lz = transfer.log_zr_lattice(g.n, g.ei, g.ej, Jt, bt, W, s_t, g.Lx)
    db_ref = torch.stack([torch.autograd.grad(lz[b], bt, retain_graph=True)[0] for b in range(batch)])
    (dj_ref,) = torch.autograd.grad(lz.mean(), Jt)
    d_spins = to_dev_spins(s.reshape(-1))
    logZR = torch.empty(batch, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR)
    logq = torch.zeros(batch, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(model.params)
    dbeta = torch.empty(batch, dtype=torch.float64, device="cuda")
    dJ = torch.empty(g.m, dtype=torch.float64, device="cuda")
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, tv.FP32, grad, dbeta, dJ)
    torch.cuda.synchronize()
    assert float((logZR.cpu() - lz.detach()).abs().max()) / g.n <= TOL_FP32
    assert float((dbeta.cpu() - db_ref).abs().max()) <= 2e-5 * float(db_ref.abs().max())
    assert float((dJ.cpu() - dj_ref).abs().max()) <= 2e-5 * max(1.0, float(dj_ref.abs().max()))
    # d/dJ alone (no d/dbeta requested) is the same launch without the per-sample output
    dJ2 = torch.empty_like(dJ)
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, tv.FP32, grad, None, dJ2)
    torch.cuda.synchronize()
    assert torch.equal(dJ, dJ2)
    # and d/dbeta alone: the same per-sample values, no bond sums written
    db2 = torch.empty_like(dbeta)
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, tv.FP32, grad, db2, None)
    torch.cuda.synchronize()
    assert torch.equal(dbeta, db2)


def test_full_size_launch_sampled_rows():
    # The 16x16 workload at its full batch in the launch the benchmark times;
    # the oracle replays a spread of sample indices one by one.
    w = wl.workload(2)
    model = _model(w)
    B = w.batch
    seed, step = 777, 3
    spins, logq, logZR = model.sample(B, seed, step)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([np.arange(0, B, 1021), [B - 1, B - 2, 127, 128]]))
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, p_or, u = oracle_samples(p32, D, w.hidden, seed, step, k, B, rows=rows)
        s_gpu = model.spins_of(spins, k, B).cpu().numpy()[rows].astype(np.float64)
        same = check_sample_agreement(s_gpu, s_or.numpy(), u, p_or.numpy(), max_flip_frac=0.1)
        lq_or = made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, w.hidden, s_or)
        lz_or = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, beta, W, s_or, g.Lx)
        m = torch.as_tensor(same)
        lq = logq[k * B:(k + 1) * B].cpu().double()[rows]
        lz = logZR[k * B:(k + 1) * B].cpu()[rows]
        assert float((lq[m] - lq_or[m]).abs().max()) / g.n <= TOL_FP32
        assert float((lz[m] - lz_or[m]).abs().max()) / g.n <= TOL_FP32


@pytest.mark.parametrize("shape", [0, 1])
def test_full_size_adjoint_sampled_rows_and_identity(shape):
    # The strip adjoint at the full 16x16 batch (5 x 16384 samples; the
    # planner's launch shape, and one warp per strip): d/dbeta of sampled rows
    # against FP64 autograd of the oracle, and for the batch-mean d/dJ the identity
    #   sum_e J_e dlogZR/dJ_e = beta * mean_b dlogZR/dbeta   (Eq. 4: weights depend on beta J only)
    w = wl.workload(2)
    model = _model(w)
    model.ctx.set_tuning((0, 0, 0, shape, 0, 0))
    B = w.batch
    seed, step = 778, 4
    spins, logq, logZR = model.sample(B, seed, step)
    grad = torch.empty_like(model.params)
    dbeta = torch.empty(model.n * B, dtype=torch.float64, device="cuda")
    dJ = torch.empty(sum(model.n_edges), dtype=torch.float64, device="cuda")
    model.ctx.backward(model.betas, B, spins, logZR, logq, tv.FP32, grad, dbeta, dJ)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([np.arange(0, B, 2039), [B - 1, 95, 96, 127, 128]]))
    eo = 0
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, p_or, u = oracle_samples(p32, D, w.hidden, seed, step, k, B, rows=rows)
        s_gpu = model.spins_of(spins, k, B).cpu().numpy()[rows].astype(np.float64)
        same = check_sample_agreement(s_gpu, s_or.numpy(), u, p_or.numpy(), max_flip_frac=0.1)
        bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        lz = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, bt, W, s_or, g.Lx)
        db_or = torch.stack([torch.autograd.grad(lz[i], bt, retain_graph=True)[0] for i in range(len(rows))])
        db = dbeta[k * B:(k + 1) * B].cpu()[rows]
        m = torch.as_tensor(same)
        assert float((db[m] - db_or[m]).abs().max()) <= 2e-5 * float(db_or.abs().max())
        lhs = float((torch.as_tensor(g.J) * dJ[eo:eo + g.m].cpu()).sum())
        rhs = beta * float(dbeta[k * B:(k + 1) * B].mean())
        assert abs(lhs - rhs) <= 1e-5 * max(1.0, abs(rhs))
        eo += g.m


@pytest.mark.parametrize("prec,overlap,shape", [(tv.FP32, 2, 0), (tv.BF16, 2, 1), (tv.BF16, 2, 96), (tv.BF16, 1, 1)])
def test_sample_contract_adjoint_equals_separate_calls(prec, overlap, shape):
    # one pass (sampling, log Z_R from the adjoint's forward sweep, d/dbeta,
    # d/dJ), with the overlapped side-stream schedule on (2) or off (1) and
    # the adjoint's launch shape, against sample_and_contract + contract +
    # backward on the same draw
    w = wl.workload(2)
    model = _model(w, n_inst=3)
    model.ctx.set_tuning((0, 0, 0, shape, 0, overlap))
    B = 1000
    spins, logq, logZR = model.buffers(B)
    dbeta = torch.empty(model.n * B, dtype=torch.float64, device="cuda")
    dJ = torch.empty(sum(model.n_edges), dtype=torch.float64, device="cuda")
    model.ctx.sample_contract_adjoint(model.betas, B, 31, 2, prec, spins, logq, logZR, dbeta, dJ)
    s2, lq2, lz2 = model.sample(B, 31, 2, precision=prec)
    lz3 = torch.empty_like(lz2)
    model.ctx.contract(model.betas, B, s2, tv.FP32, lz3)
    db2, dJ2 = torch.empty_like(dbeta), torch.empty_like(dJ)
    model.ctx.backward(model.betas, B, s2, lz2, lq2, prec, torch.empty_like(model.params), db2, dJ2)
    torch.cuda.synchronize()
    assert torch.equal(spins, s2) and torch.equal(logq, lq2)
    assert torch.equal(logZR, lz2) and torch.equal(logZR, lz3)  # same forward arithmetic
    assert torch.equal(dbeta, db2) and torch.equal(dJ, dJ2)


def test_train_step_runs_and_adam_matches_oracle():
    w = wl.workload(1)
    model = _model(w)
    p0 = model.params.cpu().numpy().astype(np.float64)
    B = 512
    spins, logq, logZR = model.sample(B, 1, 0)
    grad = torch.empty_like(model.params)
    model.ctx.backward(model.betas, B, spins, logZR, logq, tv.FP32, grad)
    g = grad.cpu().numpy().astype(np.float64)
    m = torch.zeros_like(model.params)
    v = torch.zeros_like(model.params)
    for t in (1, 2):
        model.ctx.adam(model.params, grad, m, v, 0.01, 0.9, 0.999, 1e-8, t)
    torch.cuda.synchronize()
    pr, mr, vr = est.adam_step(p0, g, np.zeros_like(g), np.zeros_like(g), 1)
    pr, mr, vr = est.adam_step(pr, g, mr, vr, 2)
    assert np.abs(model.params.cpu().numpy() - pr).max() < 1e-6


@pytest.mark.parametrize("cfg,batch,prec", [(1, 300, tv.TF32), (2, 200, tv.TF32), (2, 200, tv.BF16),
                                            (3, 130, tv.TF32), (3, 130, tv.BF16)])
def test_tensor_core_backward_matches_oracle(cfg, batch, prec):
    """TF32 / BF16 tcgen05 backward vs the FP64 oracle gradient on the same samples.
    Reduced-precision operands: the error bound is relative to the largest
    gradient entry, and the direction must agree (cosine similarity)."""
    from oracle import dense

    w = wl.workload(cfg)
    model = _model(w, scale=1.5)
    s_all, lq_all, lz_all, ref = [], [], [], []
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        th = torch.as_tensor(p32, dtype=torch.float64)
        s_or, _, _ = oracle_samples(p32, D, w.hidden, 7, 1, k, batch)
        lq = made.log_q(th, D, w.hidden, s_or).float().double()
        if g.topology == wl.DENSE:
            lz = dense.log_zr_dense(g.n, g.ei, g.ej, g.J, beta, W, s_or)
        else:
            lz = _oracle_logzr(g, W, s_or, beta)
        wts = est.reinforce_weights(lz, lq, beta)
        ref.append(est.surrogate_grad(p32.astype(np.float64), D, w.hidden, s_or, wts))
        s_all.append(s_or.numpy().reshape(-1))
        lq_all.append(lq.numpy())
        lz_all.append(lz.detach().numpy())
    d_spins = to_dev_spins(np.concatenate(s_all))
    logq = torch.as_tensor(np.concatenate(lq_all), dtype=torch.float32).cuda()
    logZR = torch.as_tensor(np.concatenate(lz_all)).cuda()
    grad = torch.full_like(model.params, float("nan"))
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, prec, grad)
    torch.cuda.synchronize()
    # reduced-precision operands: near-zero ReLU pre-activations can flip their
    # mask, so the bound is on the relative Frobenius error and the direction
    fro_max = 3e-2 if prec == tv.TF32 else 1e-1
    cos_min = 0.999 if prec == tv.TF32 else 0.99
    for k in range(model.n):
        gk = grad[model.offsets[k]:model.offsets[k + 1]].cpu().double()
        assert torch.isfinite(gk).all()
        fro = float((gk - ref[k]).norm() / ref[k].norm())
        cos = float(torch.nn.functional.cosine_similarity(gk, ref[k], dim=0))
        print(f"cfg{cfg} inst{k} prec{prec}: rel Frobenius err = {fro:.2e}, cos = {cos:.6f}")
        assert fro <= fro_max
        assert cos >= cos_min
        # entries outside the MADE masks are exactly zero
        off = torch.as_tensor(_param_mask(model.D[k], w.hidden) == 0)
        assert torch.equal(gk[off], torch.zeros_like(gk[off]))


TOL_RED = 1e-3  # |delta log q| / N in the reduced-precision modes


@pytest.mark.parametrize("group", [4, 6, 8, 12, 16, 32])
def test_bf16_tensor_core_sampler_log_prob_matches_oracle(group):
    # every plan of both tensor-core sampler forms (the autotuner picks one)
    w = wl.workload(2)
    model = _model(w, scale=1.5)
    model.ctx.set_tuning((0, 0, 0, 0, group, 0))
    batch = 96
    s_all, refs = [], []
    for k in range(model.n):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, model.D[k], w.hidden, 3, 0, k, batch)
        s_all.append(s_or.numpy().reshape(-1))
        refs.append(made.log_q(torch.as_tensor(p32, dtype=torch.float64), model.D[k], w.hidden, s_or))
    d_spins = to_dev_spins(np.concatenate(s_all))
    logq = torch.empty(model.n * batch, dtype=torch.float32, device="cuda")
    model.ctx.profile(True)
    model.ctx.log_prob(batch, d_spins, logq, tv.BF16)
    torch.cuda.synchronize()
    assert "log_prob_tc" in model.ctx.profile_read()  # the tensor-core path ran
    model.ctx.profile(False)
    for k in range(model.n):
        err = float((logq[k * batch:(k + 1) * batch].cpu().double() - refs[k]).abs().max())
        print(f"bf16 log q, instance {k}: max |delta| / N = {err / w.graphs[k].n:.2e}")
        assert err / w.graphs[k].n <= TOL_RED


def test_bf16_sampler_self_consistent_and_contracts_exactly():
    w = wl.workload(2)
    model = _model(w, n_inst=2)
    B = 300
    spins, logq, logZR = model.sample(B, 9, 4, precision=tv.BF16)
    lq2 = torch.empty_like(logq)
    model.ctx.log_prob(B, spins, lq2, tv.BF16)
    lz2 = torch.empty_like(logZR)
    model.ctx.contract(model.betas, B, spins, tv.FP32, lz2)
    torch.cuda.synchronize()
    assert torch.allclose(logq, lq2, atol=1e-5, rtol=0)  # same arithmetic, teacher-forced
    assert torch.equal(logZR, lz2)  # contraction stays FP32


def test_bf16_sampler_distribution_matches_oracle_marginal():
    from paper_2504_12037_gb300.model import TNVAN

    g = wl.sk(16, 77)
    W = np.arange(16, dtype=np.int32)  # empty remainder: only the sampler matters
    hidden = [32, 32]
    model = TNVAN([g], [W], hidden, [1.0], seed=4, init_scale=2.0)
    B = 200000
    spins, logq, _ = model.sample(B, 1234, 0, precision=tv.BF16)
    s = model.spins_of(spins, 0, B)[:, :4].cpu().numpy()
    idx = (((1 - s) // 2) * (2 ** np.arange(4))).sum(1)
    counts = np.bincount(idx, minlength=16).astype(float)
    # exact marginal of the first four spins: prod_{i<4} q(s_i | s_<i)
    th = torch.as_tensor(model.params.cpu().numpy().astype(np.float64))
    from oracle import ising
    X4 = ising.all_configs(4)
    full = torch.zeros(16, 16, dtype=torch.float64)
    full[:, :4] = X4
    x = made.logits(th, 16, hidden, full)[:, :4]
    q4 = torch.exp(-torch.nn.functional.softplus(-X4 * x).sum(1)).numpy()
    chi2 = float(((counts - B * q4) ** 2 / (B * q4)).sum())
    print("chi2 (15 dof):", chi2)
    assert chi2 < 45
