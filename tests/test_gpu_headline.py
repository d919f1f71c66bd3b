"""GPU parity of the 16x16 training step at its full size, as the benchmark
runs it (autotuned launch shapes, overlapped schedule, BF16 network, captured
CUDA graph), of the step statistics, of the autograd wrapper of F_q, and of
the data-parallel split of the training step.  Every expected value comes
from the FP64 oracle on the GPU's own samples."""
import math

import numpy as np
import pytest
import torch

from oracle import estimators as est
from oracle import ising, made, transfer
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-6  # |delta log Z_R| / N, |delta log q| / N in FP32
TOL_RED = 1e-3  # |delta log q| / N in BF16


def _model(w, n_inst=None, seed=3, scale=1.0):
    from paper_2504_12037_gb300.model import TNVAN

    n = len(w.graphs) if n_inst is None else n_inst
    return TNVAN(w.graphs[:n], w.widths_sets[:n], w.hidden, w.betas[:n], seed=seed, init_scale=scale)


def _rows(B):
    # every 1021st sample plus CTA (128) and wave (2 x 152 CTAs of 128) boundaries
    extra = [0, 1, 127, 128, 255, 256, 38911, 38912, B - 2, B - 1]
    return np.unique(np.concatenate([np.arange(0, B, 1021), [r for r in extra if r < B]]))


@pytest.mark.parametrize("prec", [tv.BF16, tv.FP32])
def test_captured_full_size_step_against_oracle(prec):
    """The benchmark's step: workload 2 at 5 x 16,384 samples, autotuned, as one
    captured CUDA graph; one replay, then sampled rows of the GPU's own samples
    against the oracle (log q on the parameters the step sampled with, log Z_R,
    d log Z_R / d beta by FP64 autograd) and the step's F_q, F_IS, stderr and
    log Z_IS against the oracle's estimators over the whole batch."""
    w = wl.workload(2)
    model = _model(w)
    B = w.batch
    model.ctx.reserve(B)
    tuned = model.ctx.autotune(model.betas, B, prec)
    dbeta = torch.empty(model.n * B, dtype=torch.float64, device="cuda")
    dJ = torch.empty(sum(model.n_edges), dtype=torch.float64, device="cuda")
    cs = model.capture_train_step(B, 4711, prec, 0.01, None, dbeta, dJ)
    cs.replay()
    torch.cuda.synchronize()
    p_before = model.params.cpu().numpy().copy()
    cs.replay()
    torch.cuda.synchronize()
    spins, logq, logZR = cs.out
    stats = cs.stats.cpu().numpy()
    rows = _rows(B)
    worst = {"logq": 0.0, "logZR": 0.0, "dbeta": 0.0}
    for k in range(model.n):
        g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
        th = torch.as_tensor(p_before[model.offsets[k]:model.offsets[k + 1]].astype(np.float64))
        s = model.spins_of(spins, k, B).cpu().numpy()[rows].astype(np.float64)
        st = torch.as_tensor(s)
        lq_or = made.log_q(th, D, w.hidden, st)
        bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        lz_or = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, bt, W, st, g.Lx)
        db_or = torch.stack([torch.autograd.grad(lz_or[i], bt, retain_graph=True)[0] for i in range(len(rows))])
        lq = logq[k * B:(k + 1) * B].cpu().double()[rows]
        lz = logZR[k * B:(k + 1) * B].cpu()[rows]
        db = dbeta[k * B:(k + 1) * B].cpu()[rows]
        e_q = float((lq - lq_or).abs().max()) / g.n
        e_z = float((lz - lz_or.detach()).abs().max()) / g.n
        e_b = float((db - db_or).abs().max()) / float(db_or.abs().max())
        worst = {"logq": max(worst["logq"], e_q), "logZR": max(worst["logZR"], e_z),
                 "dbeta": max(worst["dbeta"], e_b)}
        assert e_q <= (TOL_RED if prec == tv.BF16 else TOL_FP32)
        assert e_z <= TOL_FP32
        assert e_b <= 2e-5
        # the step's Eq. 9 statistics against the oracle's estimators on the
        # whole batch the step drew
        fe = est.free_energies(logZR[k * B:(k + 1) * B].cpu(), logq[k * B:(k + 1) * B].cpu().double(), beta)
        for j, key in enumerate(("F_q", "F_IS", "stderr", "logZ_IS")):
            assert abs(stats[k, j] - fe[key]) / g.n <= 1e-9, (k, key, stats[k, j], fe[key])
        assert stats[k, 5] == 0 and stats[k, 7] == B
    print(f"prec {prec} tuning {tuned}: worst |dlogq|/N {worst['logq']:.2e}, |dlogZR|/N {worst['logZR']:.2e}, "
          f"rel d/dbeta {worst['dbeta']:.2e}")


def test_train_step_statistics_equal_free_energy():
    # the statistics reduced inside tnvan_train_step are tnvan_free_energy's
    # on the step's own buffers (same reduction, same order)
    w = wl.workload(2)
    model = _model(w, n_inst=3)
    B = 3000
    out = model.buffers(B)
    dbeta = torch.empty(model.n * B, dtype=torch.float64, device="cuda")
    for prec in (tv.BF16, tv.FP32):
        model.train_step(B, 5, 1, prec, 0.01, out, dbeta, None)
        st = model.step_stats().cpu().numpy()
        fe = model.free_energy(B, out[2], out[1])
        assert np.array_equal(st[:, :4], fe)
        assert np.all(st[:, 7] == B) and np.all(st[:, 5] == 0)


def test_free_energy_function_gradients():
    """FreeEnergyFunction (F_q as an autograd function of theta and J): its
    backward against the oracle's REINFORCE surrogate gradient (theta) and FP64
    central differences of -(1/beta) mean_b log Z_R(s_b) (J), on the samples
    its forward drew."""
    from paper_2504_12037_gb300.model import FreeEnergyFunction

    w = wl.workload(1)
    model = _model(w, scale=1.5)
    g, W, D, beta = w.graphs[0], w.widths_sets[0], model.D[0], w.betas[0]
    B, seed, step = 128, 21, 2
    params = model.params.clone().requires_grad_(True)
    J = torch.as_tensor(g.J, dtype=torch.float64, device="cuda").requires_grad_(True)
    F = FreeEnergyFunction.apply(params, J, model, B, seed, step, tv.FP32)
    F.sum().backward()
    spins, logq, logZR = model.sample(B, seed, step)  # the same draw (same seed and step)
    torch.cuda.synchronize()
    s = torch.as_tensor(model.spins_of(spins, 0, B).cpu().numpy().astype(np.float64))
    th = model.params.cpu().numpy().astype(np.float64)
    lq_or = made.log_q(torch.as_tensor(th), D, w.hidden, s)
    lz_or = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, beta, W, s)
    # forward: F_q of the batch
    fq_or = est.free_energies(lz_or, lq_or, beta)["F_q"]
    assert abs(float(F[0]) - fq_or) / g.n <= TOL_FP32
    # theta: Eq. 10 with the batch-mean baseline
    wts = est.reinforce_weights(lz_or, lq_or, beta)
    g_or = est.surrogate_grad(th, D, w.hidden, s, wts)
    g_gpu = params.grad.cpu().double()
    assert float((g_gpu - g_or).abs().max()) <= 2e-5 * float(g_or.abs().max())
    # J: central differences in FP64 of -(1/beta) mean_b log Z_R(s_b)
    h = 1e-5
    fd = np.zeros(g.m)
    for e in range(g.m):
        Jp, Jm = np.array(g.J, np.float64), np.array(g.J, np.float64)
        Jp[e] += h
        Jm[e] -= h
        fp = -float(ising.log_zr_enum(g.n, g.ei, g.ej, Jp, beta, W, s).mean()) / beta
        fm = -float(ising.log_zr_enum(g.n, g.ei, g.ej, Jm, beta, W, s).mean()) / beta
        fd[e] = (fp - fm) / (2 * h)
    gJ = J.grad.cpu().numpy()
    assert np.abs(gJ - fd).max() <= 2e-5 * max(1.0, np.abs(fd).max())


def test_data_parallel_split_step():
    """The data-parallel step on one GPU: (1) one part -- sampling with the
    adjoint, tnvan_reduce, tnvan_merge_stats of one part, tnvan_backward_stats,
    Adam -- equals tnvan_train_step (samples, statistics and gradient bit for
    bit); (2) a batch cut into two
    parts: the merged statistics equal the whole batch's (FP64 rounding) and
    the per-part gradients with the merged baseline sum to the whole batch's
    gradient (FP32 rounding)."""
    w = wl.workload(2)
    B = 4096
    for prec in (tv.BF16, tv.FP32):
        a, b = _model(w, n_inst=1, seed=8), _model(w, n_inst=1, seed=8)
        out_a, out_b = a.buffers(B), b.buffers(B)
        db_a = torch.empty(B, dtype=torch.float64, device="cuda")
        db_b = torch.empty_like(db_a)
        a.train_step(B, 99, 3, prec, 0.01, out_a, db_a, None)
        b.ctx.sample_contract_adjoint(b.betas, B, 99, 3, prec, *out_b, db_b, None)
        part = torch.empty(8, dtype=torch.float64, device="cuda")
        b.ctx.reduce(b.betas, B, out_b[2], out_b[1], part)
        merged = torch.empty(8, dtype=torch.float64, device="cuda")
        b.ctx.merge_stats(b.betas, part.view(1, 8), merged)
        b.ctx.backward_stats(b.betas, B, out_b[0], out_b[2], out_b[1], prec, b.grad)
        b.t += 1
        b.ctx.adam(b.params, b.grad, b.m, b.v, 0.01, 0.9, 0.999, 1e-8, b.t)
        torch.cuda.synchronize()
        assert all(torch.equal(x, y) for x, y in zip(out_a, out_b))
        assert torch.equal(a.grad, b.grad)
        # Adam fused into the gradient reduction vs the separate Adam kernel
        # (bias corrections formed in different precisions)
        assert torch.allclose(a.params, b.params, rtol=1e-6, atol=1e-9)
        assert torch.equal(part, merged)
        assert torch.equal(a.step_stats().view(-1), merged)
        # two parts of the same batch (samples [0, B/2) and [B/2, B))
        h = B // 2
        D = b.D[0]
        spins, logq, logZR = out_b
        parts = torch.empty(2, 8, dtype=torch.float64, device="cuda")
        b.ctx.reduce(b.betas, h, logZR[:h], logq[:h], parts[0])
        b.ctx.reduce(b.betas, h, logZR[h:], logq[h:], parts[1])
        b.ctx.merge_stats(b.betas, parts, merged)
        whole = torch.empty(8, dtype=torch.float64, device="cuda")
        b.ctx.reduce(b.betas, B, logZR, logq, whole)
        g_whole = torch.empty_like(b.grad)
        b.ctx.backward_stats(b.betas, B, spins, logZR, logq, prec, g_whole)
        b.ctx.merge_stats(b.betas, parts, merged)
        g0, g1 = torch.empty_like(b.grad), torch.empty_like(b.grad)
        b.ctx.backward_stats(b.betas, h, spins[:h * D], logZR[:h], logq[:h], prec, g0)
        b.ctx.backward_stats(b.betas, h, spins[h * D:], logZR[h:], logq[h:], prec, g1)
        torch.cuda.synchronize()
        m, wv = merged.cpu().numpy(), whole.cpu().numpy()
        for j in (0, 1, 3, 4):
            assert abs(m[j] - wv[j]) <= 1e-12 * max(1.0, abs(wv[j])), (j, m[j], wv[j])
        assert abs(m[2] - wv[2]) <= 1e-9 * wv[2] and abs(m[6] - wv[6]) <= 1e-9 * wv[6]
        assert m[7] == B and m[5] == 0
        gs = (g0 + g1).double()
        assert float((gs - g_whole.double()).abs().max()) <= 1e-4 * float(g_whole.double().abs().max())


def test_device_merge_equals_host_merge():
    # tnvan_merge_stats (device kernel) against dp.merge_stats (host, FP64) on
    # statistics rows of three parts, one of which has no finite samples
    from paper_2504_12037_gb300 import dp

    w = wl.workload(2)
    model = _model(w, n_inst=2)
    rng = np.random.default_rng(6)
    parts = []
    for p, n in enumerate((300, 0, 1100)):
        rows = []
        for k in range(model.n):
            l = rng.normal(-50 * (k + 1), 2 + p, size=max(n, 1))
            b = model.betas[k]
            lz = l.max() + np.log(np.exp(l - l.max()).sum()) - np.log(len(l))
            row = [-l.mean() / b, -lz / b, l.std(ddof=1) / (b * np.sqrt(len(l))), lz, l.mean(), 2.0, l.var(ddof=1),
                   float(n)]
            rows.append(row if n else [np.nan] * 4 + [np.nan, 5.0, np.nan, 0.0])
        parts.append(rows)
    parts = np.array(parts)
    host = dp.merge_stats(parts, model.betas)
    d_parts = torch.as_tensor(parts).cuda()
    out = torch.empty(model.n * 8, dtype=torch.float64, device="cuda")
    model.ctx.merge_stats(model.betas, d_parts, out)
    dev = out.cpu().numpy().reshape(model.n, 8)
    assert np.allclose(dev, host, rtol=1e-13, atol=0)
    assert np.all(dev[:, dp.BAD] == 9.0) and np.all(dev[:, dp.N] == 1400)
    st = model.step_stats().cpu().numpy()  # the merge became the context's statistics
    assert np.array_equal(st, dev)


@pytest.mark.parametrize("prec", [tv.BF16, tv.FP32])
def test_train_step_without_adjoint_outputs(prec):
    # a training step that asks for neither d/dbeta nor d/dJ runs only the
    # forward strip chain in its contraction pass: its samples, log q and
    # log Z_R equal those of the same step with d/dbeta requested (same
    # parameters, seed and step), log Z_R equals tnvan_contract's on those
    # samples, and sampled rows match the oracle
    w = wl.workload(2)
    B = 700  # several CTAs per instance and chunk, ragged last CTA
    a, b = _model(w, n_inst=3, seed=8), _model(w, n_inst=3, seed=8)
    out_a, out_b = a.buffers(B), b.buffers(B)
    dbeta = torch.empty(b.n * B, dtype=torch.float64, device="cuda")
    a.train_step(B, 17, 4, prec, 0.01, out_a, None, None)
    b.train_step(B, 17, 4, prec, 0.01, out_b, dbeta, None)
    torch.cuda.synchronize()
    assert torch.equal(out_a[0], out_b[0]) and torch.equal(out_a[1], out_b[1])
    assert torch.allclose(out_a[2], out_b[2], rtol=1e-12, atol=0)
    lz = torch.empty_like(out_a[2])
    a.ctx.contract(a.betas, B, out_a[0], prec, lz)
    torch.cuda.synchronize()
    assert torch.allclose(lz, out_a[2], rtol=1e-12, atol=0)
    rows = np.arange(0, B, 97)
    for k in range(a.n):
        g, W = w.graphs[k], w.widths_sets[k]
        s = torch.as_tensor(a.spins_of(out_a[0], k, B).cpu().numpy().astype(np.float64)[rows])
        ref = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, w.betas[k], W, s, g.Lx).numpy()
        err = np.abs(out_a[2][k * B:(k + 1) * B].cpu().numpy()[rows] - ref).max() / g.n
        assert err <= TOL_FP32, (k, err)
