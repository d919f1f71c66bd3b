"""GPU parity of tnvan_magnetisation (Sec. 3: magnetisation and susceptibility
from samples) against the FP64 oracle, through the C-ABI: per-sample
conditional moments E[M | s] and Var(M | s) for strip, dense and elimination
instances side by side in one context, and the importance-weighted averages.
Width-set rows and log q are seeded inputs; the oracle contracts every row
with a uniform field on R and differentiates twice."""
import math

import numpy as np
import pytest
import torch

from oracle import dense, general, transfer
from oracle import magnetisation as mg
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import to_dev_spins

pytestmark = pytest.mark.gpu


def _contract(g, W, beta, s):
    if g.topology == wl.DENSE:
        return lambda h: dense.log_zr_dense(g.n, g.ei, g.ej, g.J, beta, W, s, field=h)
    if g.topology == wl.LATTICE2D:
        return lambda h: transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, beta, W, s, g.Lx, field=h)
    return lambda h: general.log_zr_general(g.n, g.ei, g.ej, g.J, beta, W, s, field=h)


def _case(kinds):
    graphs, Ws, betas = [], [], []
    if "strips" in kinds:
        # strips of widths 1-4 with mixed-sign couplings (gauge flips), 20 rows
        graphs.append(wl.lattice(14, 20, "gauss", seed=93))
        Ws.append(wl.width_columns(14, 20, [1, 4, 8, 13]))
        betas.append(0.7)
    if "ferro" in kinds:
        # the open ferromagnet below T_c: strongly magnetised conditionals
        graphs.append(wl.lattice(12, 12, "ferro", seed=0))
        Ws.append(wl.width_columns(12, 12, wl.every_kth_column(12, 5)))
        betas.append(0.6)
    if "dense" in kinds:
        # |R| = 14 (a half with phantom spins) and |R| = 16
        for n, nw, seed in ((22, 8, 4), (24, 8, 5)):
            graphs.append(wl.sk(n, seed))
            Ws.append(np.arange(nw, dtype=np.int32))
            betas.append(1.1)
    if "general" in kinds:
        g = wl.random_regular(256, 3, 17)
        graphs.append(g)
        Ws.append(wl.greedy_width_set(g, 17))
        betas.append(1.0)
    return graphs, Ws, betas


@pytest.mark.parametrize("kinds", [("strips", "ferro"), ("dense",), ("general",), ("strips", "dense", "general")])
def test_magnetisation_matches_oracle(kinds):
    from paper_2504_12037_gb300.model import TNVAN

    graphs, Ws, betas = _case(kinds)
    batch = 160  # several tiles of every kind, ragged last tile
    model = TNVAN(graphs, Ws, [32, 32], betas, seed=5)
    rng = np.random.default_rng(len(kinds))
    s_all, lq_all, refs = [], [], []
    for g, W, beta in zip(graphs, Ws, betas):
        D = len(W)
        s = np.where(rng.random((batch, D)) < 0.5, 1.0, -1.0)
        if g.topology == wl.LATTICE2D and g.J.min() > 0:
            s[: batch // 2] = 1.0  # aligned width sets: |E[M | s]| near N
        lq = rng.normal(-D * math.log(2.0), 3.0, size=batch).astype(np.float32)
        st = torch.as_tensor(s)
        mean, var = mg.conditional_moments(_contract(g, W, beta, st), st, W, beta)
        lz = _contract(g, W, beta, st)(None).detach()
        refs.append((mean.numpy(), var.numpy(),
                     mg.magnetisation_stats(lz, torch.as_tensor(lq, dtype=torch.float64), mean, var, beta, g.n)))
        s_all.append(s.reshape(-1))
        lq_all.append(lq)
    n = len(graphs)
    d_spins = to_dev_spins(np.concatenate(s_all))
    logq = torch.as_tensor(np.concatenate(lq_all)).cuda()
    logZR = torch.empty(n * batch, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR)
    d_mean = torch.full((n * batch,), float("nan"), dtype=torch.float64, device="cuda")
    d_var = torch.full_like(d_mean, float("nan"))
    out = model.ctx.magnetisation(model.betas, batch, d_spins, logZR, logq, d_mean, d_var)
    torch.cuda.synchronize()
    mean_g, var_g = d_mean.cpu().numpy(), d_var.cpu().numpy()
    for k, (g, (m_ref, v_ref, st_ref)) in enumerate(zip(graphs, refs)):
        sl = slice(k * batch, (k + 1) * batch)
        N = g.n
        # FP32 chains: relative rounding ~1e-5 of sums bounded by N (mean) and
        # by the moments' own scale (variance)
        assert np.abs(mean_g[sl] - m_ref).max() <= 1e-5 * N, (k, np.abs(mean_g[sl] - m_ref).max())
        assert np.all(var_g[sl] >= 0.0)
        assert np.all(np.abs(var_g[sl] - v_ref) <= 1e-4 * np.maximum(v_ref, 1.0) + 1e-5 * N), k
        M1, M2, chi, M1q, M2q, ess = out[k]
        r1, r2, rchi, r1q, r2q, ress = st_ref
        assert abs(M1 - r1) <= 1e-4 * N, (k, M1, r1)
        assert abs(M2 - r2) <= 1e-4 * max(r2, N), (k, M2, r2)
        assert abs(chi - g.n ** -1 * betas_of(model, k) * (M2 - M1 * M1)) <= 1e-9 * max(abs(chi), 1.0)
        assert abs(chi - rchi) <= 1e-3 * max(abs(rchi), 1.0), (k, chi, rchi)
        assert abs(M1q - r1q) <= 1e-5 * N and abs(M2q - r2q) <= 1e-5 * max(r2q, N)
        assert abs(ess - ress) <= 1e-4 * ress and 1.0 <= ess <= batch
    # the moments alone (workspace outputs) give the same averages
    out2 = model.ctx.magnetisation(model.betas, batch, d_spins, logZR, logq)
    torch.cuda.synchronize()
    assert np.array_equal(out, out2)


def betas_of(model, k):
    return float(model.betas[k])


def test_magnetisation_zero_field_symmetry_and_uniform_weights():
    # flipping every width-set spin of a zero-field instance flips E[M | s]
    # and keeps Var(M | s); equal l_b give ESS = B and the q-averages
    from paper_2504_12037_gb300.model import TNVAN

    graphs, Ws, betas = _case(("strips", "dense", "general"))
    model = TNVAN(graphs, Ws, [32, 32], betas, seed=6)
    B = 96
    rng = np.random.default_rng(9)
    s = [np.where(rng.random((B, len(W))) < 0.5, 1.0, -1.0) for W in Ws]
    both = [np.concatenate([x, -x]) for x in s]
    d_spins = to_dev_spins(np.concatenate([x.reshape(-1) for x in both]))
    n = len(graphs)
    logZR = torch.empty(n * 2 * B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, 2 * B, d_spins, tv.FP32, logZR)
    logq = logZR.float()
    mean = torch.empty(n * 2 * B, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    out = model.ctx.magnetisation(model.betas, 2 * B, d_spins, logZR, logq, mean, var)
    torch.cuda.synchronize()
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    for k in range(n):
        a, b = slice(2 * k * B, 2 * k * B + B), slice(2 * k * B + B, 2 * (k + 1) * B)
        assert np.abs(mean[a] + mean[b]).max() <= 1e-5 * graphs[k].n
        assert np.abs(var[a] - var[b]).max() <= 1e-4 * max(1.0, float(np.abs(var[a]).max()))
        M1, M2, chi, M1q, M2q, ess = out[k]
        assert abs(ess - 2 * B) <= 1e-3 * 2 * B  # l_b = 0 up to the FP32 rounding of log q
        assert abs(M1q) <= 1e-5 * graphs[k].n
        assert abs(M2q - float((mean[2 * k * B:2 * (k + 1) * B] ** 2 + var[2 * k * B:2 * (k + 1) * B]).mean())) \
            <= 1e-9 * M2q
