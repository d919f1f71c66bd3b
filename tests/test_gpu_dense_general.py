"""GPU parity of the dense (SK) and general-component (random regular graph)
contractions, and of the multi-instance lattice workload, through the C-ABI."""
import numpy as np
import pytest
import torch

from oracle import dense, general, ising, made, transfer
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import check_sample_agreement, oracle_samples, to_dev_spins

pytestmark = pytest.mark.gpu
TOL_FP32 = 1e-6


def _model(graphs, Ws, hidden, betas, seed=3, scale=1.5):
    from paper_2504_12037_gb300.model import TNVAN

    return TNVAN(graphs, Ws, hidden, betas, seed=seed, init_scale=scale)


def _oracle_logzr(g, W, s, beta, J=None):
    J = g.J if J is None else J
    if g.topology == wl.DENSE:
        return dense.log_zr_dense(g.n, g.ei, g.ej, J, beta, W, s)
    if g.topology == wl.LATTICE2D:
        return transfer.log_zr_lattice(g.n, g.ei, g.ej, J, beta, W, s, g.Lx)
    return general.log_zr_general(g.n, g.ei, g.ej, J, beta, W, s)


def _parity(model, graphs, Ws, hidden, betas, batch, seed=11, step=2, check_db=True):
    s_all, lq_ref, lz_ref, db_ref = [], [], [], []
    for k in range(model.n):
        g, W, D, beta = graphs[k], Ws[k], model.D[k], betas[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, D, hidden, seed, step, k, batch)
        s_all.append(s_or.numpy().reshape(-1))
        lq_ref.append(made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, hidden, s_or))
        bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        lz = _oracle_logzr(g, W, s_or, bt)
        lz_ref.append(lz.detach())
        if check_db:
            db_ref.append(torch.stack([torch.autograd.grad(lz[b], bt, retain_graph=True)[0] for b in range(batch)]))
    d_spins = to_dev_spins(np.concatenate(s_all))
    n = model.n
    logq = torch.empty(n * batch, dtype=torch.float32, device="cuda")
    logZR = torch.empty(n * batch, dtype=torch.float64, device="cuda")
    dbeta = torch.empty(n * batch, dtype=torch.float64, device="cuda")
    model.ctx.log_prob(batch, d_spins, logq)
    model.ctx.contract(model.betas, batch, d_spins, tv.FP32, logZR, dbeta if check_db else None)
    torch.cuda.synchronize()
    for k in range(n):
        N = graphs[k].n
        sl = slice(k * batch, (k + 1) * batch)
        assert float((logq[sl].cpu().double() - lq_ref[k]).abs().max()) / N <= TOL_FP32
        assert float((logZR[sl].cpu() - lz_ref[k]).abs().max()) / N <= TOL_FP32
        if check_db:
            ref = db_ref[k]
            assert float((dbeta[sl].cpu() - ref).abs().max()) <= 2e-5 * max(1.0, float(ref.abs().max()))
    return d_spins


def test_sk_dense_block_parity():
    w = wl.workload(3)
    model = _model(w.graphs, w.widths_sets, w.hidden, w.betas)
    _parity(model, w.graphs, w.widths_sets, w.hidden, w.betas, batch=40)
    assert model.ctx.instance_info(0)["kind"] == 1


def test_sk_dense_block_small_remainders():
    # |R| = 10 (phantom padding in both halves), |R| = 3 and |R| = 0
    graphs, Ws = [], []
    for n, nw, seed in [(20, 10, 1), (11, 8, 2), (9, 9, 3)]:
        g = wl.sk(n, seed)
        graphs.append(g)
        Ws.append(np.random.default_rng(seed).permutation(n)[:nw].astype(np.int32))
    betas = [0.7, 1.3, 2.0]
    model = _model(graphs, Ws, [12], betas)
    for k in range(3):
        assert model.ctx.instance_info(k)["kind"] == 1
    _parity(model, graphs, Ws, [12], betas, batch=33)


def test_sk_dense_adjoint_dJ():
    g = wl.sk(18, 4)
    W = np.arange(6, 18, dtype=np.int32)
    model = _model([g], [W], [16], [1.1])
    B = 24
    p32 = model.params.cpu().numpy()
    s_or, _, _ = oracle_samples(p32, 12, [16], 3, 0, 0, B)
    Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lz = dense.log_zr_dense(g.n, g.ei, g.ej, Jt, 1.1, W, s_or)
    (ref,) = torch.autograd.grad(lz.mean(), Jt)
    d_spins = to_dev_spins(s_or.numpy().reshape(-1))
    logZR = torch.empty(B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, logZR)
    dJ = torch.empty(g.m, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(model.params)
    model.ctx.backward(model.betas, B, d_spins, logZR, torch.zeros(B, dtype=torch.float32, device="cuda"),
                       tv.FP32, grad, None, dJ)
    torch.cuda.synchronize()
    assert float((dJ.cpu() - ref).abs().max()) <= 2e-5 * max(1.0, float(ref.abs().max()))


def test_rrg_general_components_parity():
    w = wl.workload(4)
    model = _model(w.graphs, w.widths_sets, w.hidden, w.betas)
    info = model.ctx.instance_info(0)
    assert info["kind"] == 2 and info["max_width"] <= 8 and info["max_component"] <= 40
    _parity(model, w.graphs, w.widths_sets, w.hidden, w.betas, batch=24)


@pytest.mark.parametrize("with_db", [False, True])
def test_rrg_component_tables_large_batch(with_db):
    # components with at most 12 width-set neighbours are tabulated over their
    # boundary configurations (log Z_c and d/dbeta at the call's beta) when the
    # tables are smaller than the batch; the large batch (tables) against the
    # same rows contracted as a small batch (elimination per sample) and, on
    # sampled rows, against the oracle
    w = wl.workload(4)
    g, W, beta = w.graphs[0], w.widths_sets[0], w.betas[0]
    model = _model(w.graphs, w.widths_sets, w.hidden, w.betas)
    D = model.D[0]
    B = 1 << 16
    s = np.where(np.random.default_rng(31).random((B, D)) < 0.5, 1, -1).astype(np.int8)
    d_spins = to_dev_spins(s.reshape(-1))
    logZR = torch.empty(B, dtype=torch.float64, device="cuda")
    dbeta = torch.empty(B, dtype=torch.float64, device="cuda") if with_db else None
    model.ctx.profile(True)
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, logZR, dbeta)
    torch.cuda.synchronize()
    model.ctx.profile(False)
    assert "general_tables" in model.ctx.profile_read()
    n_small = 24
    lz_small = torch.empty(n_small, dtype=torch.float64, device="cuda")
    db_small = torch.empty(n_small, dtype=torch.float64, device="cuda") if with_db else None
    model.ctx.profile(True)
    model.ctx.contract(model.betas, n_small, to_dev_spins(s[:n_small].reshape(-1)), tv.FP32, lz_small, db_small)
    torch.cuda.synchronize()
    model.ctx.profile(False)
    model.ctx.profile_read()
    assert float((logZR[:n_small] - lz_small).abs().max()) <= 1e-9 * float(lz_small.abs().max())
    if with_db:
        assert float((dbeta[:n_small] - db_small).abs().max()) <= 1e-6 * max(1.0, float(db_small.abs().max()))
    rows = [0, 1, 2, 777, 4096, 30001, B - 2, B - 1]
    s_or = torch.as_tensor(s[rows].astype(np.float64))
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    lz = general.log_zr_general(g.n, g.ei, g.ej, g.J, bt, W, s_or)
    assert float((logZR[rows].cpu() - lz.detach()).abs().max()) / g.n <= TOL_FP32
    if with_db:
        db_ref = torch.stack([torch.autograd.grad(lz[i], bt, retain_graph=True)[0] for i in range(len(rows))])
        assert float((dbeta[rows].cpu() - db_ref).abs().max()) <= 2e-5 * max(1.0, float(db_ref.abs().max()))


def test_general_small_graphs_against_enumeration():
    graphs = [wl.random_regular(20, 3, 7), wl.random_regular(24, 4, 8, "gauss"), wl.lattice(5, 4, "gauss", 9)]
    graphs[2].topology = wl.GENERAL  # a lattice contracted as a general graph
    Ws = [np.array([0, 5, 9, 13], np.int32), np.array([1, 2, 3, 10, 17, 20], np.int32),
          np.array([2, 7, 12, 17, 6], np.int32)]
    betas = [1.0, 0.6, 0.9]
    model = _model(graphs, Ws, [10], betas)
    s_all, refs = [], []
    B = 19
    for k in range(3):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, len(Ws[k]), [10], 5, 1, k, B)
        s_all.append(s_or.numpy().reshape(-1))
        refs.append(ising.log_zr_enum(graphs[k].n, graphs[k].ei, graphs[k].ej, graphs[k].J, betas[k], Ws[k], s_or))
    d_spins = to_dev_spins(np.concatenate(s_all))
    logZR = torch.empty(3 * B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, logZR)
    torch.cuda.synchronize()
    for k in range(3):
        assert float((logZR[k * B:(k + 1) * B].cpu() - refs[k]).abs().max()) / graphs[k].n <= TOL_FP32


@pytest.mark.parametrize("which", ["rrg_workload", "small_graphs"])
def test_general_adjoint_dJ_matches_oracle(which):
    if which == "rrg_workload":
        w = wl.workload(4)
        graphs, Ws, betas, hidden = w.graphs, w.widths_sets, w.betas, w.hidden
    else:
        g1 = wl.random_regular(20, 3, 7)
        g2 = wl.lattice(5, 4, "gauss", 9)
        g2.topology = wl.GENERAL
        graphs = [g1, g2]
        Ws = [np.array([0, 5, 9, 13], np.int32), np.array([2, 7, 12, 17, 6], np.int32)]
        betas, hidden = [1.0, 0.7], [10]
    model = _model(graphs, Ws, hidden, betas)
    B = 20
    s_all, refs = [], []
    for k in range(model.n):
        g = graphs[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, model.D[k], hidden, 3, 0, k, B)
        s_all.append(s_or.numpy().reshape(-1))
        Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
        lz = general.log_zr_general(g.n, g.ei, g.ej, Jt, betas[k], Ws[k], s_or, enum_max=0)
        (ref,) = torch.autograd.grad(lz.mean(), Jt)
        refs.append(ref)
    d_spins = to_dev_spins(np.concatenate(s_all))
    n = model.n
    logZR = torch.empty(n * B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, logZR)
    dJ = torch.empty(sum(g.m for g in graphs), dtype=torch.float64, device="cuda")
    grad = torch.empty_like(model.params)
    model.ctx.backward(model.betas, B, d_spins, logZR, torch.zeros(n * B, dtype=torch.float32, device="cuda"),
                       tv.FP32, grad, None, dJ)
    torch.cuda.synchronize()
    off = 0
    for k in range(n):
        m = graphs[k].m
        got = dJ[off:off + m].cpu()
        assert float((got - refs[k]).abs().max()) <= 2e-5 * max(1.0, float(refs[k].abs().max()))
        off += m


def test_multi_instance_lattice_sizes_parity():
    w = wl.workload(5, n_instances=64)
    sizes = [g.Lx for g in w.graphs]
    pick = [sizes.index(L) for L in (8, 12, 16, 24, 32)]
    graphs = [w.graphs[i] for i in pick]
    Ws = [w.widths_sets[i] for i in pick]
    betas = [w.betas[i] for i in pick]
    model = _model(graphs, Ws, w.hidden, betas)
    assert [model.D[k] for k in range(5)] == [16, 36, 64, 144, 256]
    B = 6
    _parity(model, graphs, Ws, w.hidden, betas, batch=B, check_db=True)
    # sampler replay across all five sizes in one launch
    spins, logq, logZR = model.sample(B, 21, 9)
    torch.cuda.synchronize()
    for k in range(5):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, p_or, u = oracle_samples(p32, model.D[k], w.hidden, 21, 9, k, B)
        check_sample_agreement(model.spins_of(spins, k, B).cpu().numpy().astype(float), s_or.numpy(), u,
                               p_or.numpy(), max_flip_frac=0.34)


def test_sampler_replay_sk_and_rrg():
    for cfg in (3, 4):
        w = wl.workload(cfg)
        model = _model(w.graphs, w.widths_sets, w.hidden, w.betas)
        B = 64
        spins, logq, logZR = model.sample(B, 5, 1)
        torch.cuda.synchronize()
        for k in range(model.n):
            g, W, D, beta = w.graphs[k], w.widths_sets[k], model.D[k], w.betas[k]
            p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
            s_or, p_or, u = oracle_samples(p32, D, w.hidden, 5, 1, k, B)
            same = check_sample_agreement(model.spins_of(spins, k, B).cpu().numpy().astype(float), s_or.numpy(),
                                          u, p_or.numpy(), max_flip_frac=0.05)
            m = torch.as_tensor(same)
            lz = _oracle_logzr(g, W, s_or, beta)
            assert float((logZR[k * B:(k + 1) * B].cpu()[m] - lz[m]).abs().max()) / g.n <= TOL_FP32


@pytest.mark.parametrize("case", ["sk_workload", "small_remainders", "wide_width_sets"])
def test_dense_block_bf16_tensor_cores(case):
    # width sets of 48 (the SK workload), 8 to 10 and 70 to 84 spins: the W-side
    # terms take the unrolled shared-memory form up to 64 spins, global loads beyond
    if case == "sk_workload":
        w = wl.workload(3)
        graphs, Ws, betas = w.graphs, w.widths_sets, w.betas
    elif case == "wide_width_sets":
        graphs, Ws = [], []
        for n, seed in [(86, 4), (100, 5)]:
            graphs.append(wl.sk(n, seed))
            Ws.append(np.random.default_rng(seed).permutation(n)[:n - 16].astype(np.int32))
        betas = [0.9, 1.4]
    else:
        graphs, Ws = [], []
        for n, nw, seed in [(20, 10, 1), (11, 8, 2), (9, 9, 3)]:
            graphs.append(wl.sk(n, seed))
            Ws.append(np.random.default_rng(seed).permutation(n)[:nw].astype(np.int32))
        betas = [0.7, 1.3, 2.0]
    model = _model(graphs, Ws, [16], betas)
    B = 300  # three 128-sample tiles, the last one ragged
    s_all, refs = [], []
    for k in range(model.n):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, model.D[k], [16], 8, 0, k, B)
        s_all.append(s_or.numpy().reshape(-1))
        refs.append(dense.log_zr_dense(graphs[k].n, graphs[k].ei, graphs[k].ej, graphs[k].J, betas[k], Ws[k], s_or))
    d_spins = to_dev_spins(np.concatenate(s_all))
    logZR = torch.empty(model.n * B, dtype=torch.float64, device="cuda")
    model.ctx.profile(True)
    model.ctx.contract(model.betas, B, d_spins, tv.BF16, logZR)
    torch.cuda.synchronize()
    model.ctx.profile(False)
    for k in range(model.n):
        err = float((logZR[k * B:(k + 1) * B].cpu() - refs[k]).abs().max()) / graphs[k].n
        print(f"{case} instance {k}: max |delta log Z_R| / N = {err:.2e}")
        assert err <= 1e-3
