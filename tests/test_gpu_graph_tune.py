"""CUDA-graph capture of the sampling + contraction + backward calls with a
device step counter, and the autotuner (GPU)."""
import numpy as np
import pytest
import torch

from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _model(cfg, n=None):
    from paper_2504_12037_gb300.model import TNVAN

    w = wl.workload(cfg)
    n = len(w.graphs) if n is None else n
    return w, TNVAN(w.graphs[:n], w.widths_sets[:n], w.hidden, w.betas[:n], seed=2)


@pytest.mark.parametrize("prec", [tv.FP32, tv.BF16])
def test_graph_replay_matches_eager_and_advances(prec):
    w, m = _model(2, n=2)
    B = 1000
    m.ctx.reserve(B)
    out = m.buffers(B)
    grad = torch.empty_like(m.params)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.ctx.set_step_counter(counter)

    def step():
        m.ctx.sample_and_contract(m.betas, B, 77, 0, prec, *out)
        m.ctx.backward(m.betas, B, out[0], out[2], out[1], prec, grad)

    step()  # warm-up outside capture (workspaces, descriptors)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
        counter.add_(1)
    counter.fill_(5)
    g.replay()
    torch.cuda.synchronize()
    spins_g, logq_g, lz_g = (x.clone() for x in out)
    grad_g = grad.clone()
    assert int(counter.item()) == 6
    g.replay()
    torch.cuda.synchronize()
    assert not torch.equal(out[0], spins_g)  # a new step, new draws
    # eager call with the same effective step (counter 5 + host step 0)
    m.ctx.set_step_counter(None)
    ref = m.buffers(B)
    m.ctx.sample_and_contract(m.betas, B, 77, 5, prec, *ref)
    grad_e = torch.empty_like(grad)
    m.ctx.backward(m.betas, B, ref[0], ref[2], ref[1], prec, grad_e)
    torch.cuda.synchronize()
    assert torch.equal(ref[0], spins_g)
    assert torch.equal(ref[1], logq_g)
    assert torch.equal(ref[2], lz_g)
    assert torch.allclose(grad_e, grad_g, rtol=0, atol=0)


def test_autotune_picks_valid_shapes_and_results_unchanged():
    w, m = _model(2, n=2)
    B = 2048
    out0 = m.buffers(B)
    m.ctx.sample_and_contract(m.betas, B, 3, 1, tv.FP32, *out0)
    torch.cuda.synchronize()
    choice = m.ctx.autotune(m.betas, B, tv.FP32)
    assert choice[0] in (16, 32, 64) and choice[1] in (32, 64, 128) and choice[3] in (1, 32, 64, 96, 128)
    out1 = m.buffers(B)
    m.ctx.sample_and_contract(m.betas, B, 3, 1, tv.FP32, *out1)
    torch.cuda.synchronize()
    # launch shapes change the schedule, not the arithmetic per sample
    assert torch.equal(out0[0], out1[0])
    assert torch.allclose(out0[1], out1[1], rtol=0, atol=1e-5)
    assert torch.equal(out0[2], out1[2])
    p0 = m.params.clone()
    choice_bf = m.ctx.autotune(m.betas, B, tv.BF16)
    torch.cuda.synchronize()
    assert torch.equal(m.params, p0)  # whole training steps are timed with the networks held fixed
    assert choice_bf[2] >= 1 and choice_bf[4] in (4, 6, 8, 12, 16, 32) and choice_bf[5] in (1, 2)
    m.ctx.set_tuning(choice_bf)  # round trip
    with pytest.raises(tv.TnvanError):
        m.ctx.set_tuning((0, 0, 0, 0, 5, 0))


def test_captured_train_step_matches_eager_steps():
    # model.capture_train_step: replay k draws Philox step 1 + k with Adam's
    # t = 2 + k (counter on the device); the eager step with the same step and
    # t gives the same samples and, up to the bias corrections' rounding (formed
    # on the device from FP32 betas), the same parameters
    w = wl.workload(2)
    from paper_2504_12037_gb300.model import TNVAN

    B = 1000
    mk = lambda: TNVAN(w.graphs[:2], w.widths_sets[:2], w.hidden, w.betas[:2], seed=3)
    a, b = mk(), mk()
    dba = torch.empty(2 * B, dtype=torch.float64, device="cuda")
    dja = torch.empty(sum(a.n_edges), dtype=torch.float64, device="cuda")
    dbb, djb = torch.empty_like(dba), torch.empty_like(dja)
    outa = a.buffers(B)
    a.train_step(B, 9, 0, tv.BF16, 0.01, outa, dba, dja)
    a.train_step(B, 9, 1, tv.BF16, 0.01, outa, dba, dja)
    torch.cuda.synchronize()
    cs = b.capture_train_step(B, 9, tv.BF16, 0.01, None, dbb, djb)  # takes the eager step 0
    cs.replay()
    torch.cuda.synchronize()
    assert torch.equal(cs.out[0], outa[0]) and torch.equal(cs.out[2], outa[2])
    assert torch.equal(djb, dja) and torch.equal(dbb, dba)
    assert b.t == a.t == 2
    assert torch.allclose(a.params, b.params, rtol=1e-5, atol=1e-7)
    s1 = cs.out[0].clone()
    cs.replay()  # the next step: fresh draws
    torch.cuda.synchronize()
    assert b.t == 3 and not torch.equal(cs.out[0], s1)


@pytest.mark.parametrize("precision", [tv.BF16, tv.FP32])
def test_fused_train_step_matches_separate_calls(precision):
    # tnvan_train_step (one pack, gradient reduction and Adam in one kernel,
    # Adam on the networks' own parameters) against sample_contract_adjoint +
    # backward + adam: the same samples, contraction, adjoint and gradient,
    # and the same parameters and moments after Adam
    w = wl.workload(2)
    from paper_2504_12037_gb300.model import TNVAN

    B = 700
    mk = lambda: TNVAN(w.graphs[:3], w.widths_sets[:3], w.hidden, w.betas[:3], seed=4)
    a, b = mk(), mk()
    dba = torch.empty(3 * B, dtype=torch.float64, device="cuda")
    dja = torch.empty(sum(a.n_edges), dtype=torch.float64, device="cuda")
    dbb, djb = torch.empty_like(dba), torch.empty_like(dja)
    outa, outb = a.buffers(B), b.buffers(B)
    for step in range(2):
        a.train_step(B, 21, step, precision, 0.01, outa, dba, dja)
        b.train_step_separate(B, 21, step, precision, 0.01, outb, dbb, djb)
        torch.cuda.synchronize()
        for x, y in zip(outa, outb):
            assert torch.equal(x, y)
        assert torch.equal(dba, dbb) and torch.equal(dja, djb)
        assert torch.equal(a.grad, b.grad)
        for x, y in ((a.params, b.params), (a.m, b.m), (a.v, b.v)):
            assert torch.allclose(x, y, rtol=1e-6, atol=1e-9)
            y.copy_(x)  # the next step starts from one state (b's networks are views of b.params)
    assert a.t == b.t == 2
    assert not torch.equal(a.params, mk().params)  # Adam moved the registered parameters
    # the combined pass with d/dbeta only (no d/dJ) gives the same per-sample values
    sp1, lq1, lz1 = a.buffers(B)
    a.ctx.sample_contract_adjoint(a.betas, B, 21, 7, precision, sp1, lq1, lz1, dba, dja)
    sp2, lq2, lz2 = a.buffers(B)
    db_only = torch.empty_like(dba)
    a.ctx.sample_contract_adjoint(a.betas, B, 21, 7, precision, sp2, lq2, lz2, db_only, None)
    torch.cuda.synchronize()
    assert torch.equal(sp1, sp2) and torch.equal(lz1, lz2) and torch.equal(dba, db_only)


@pytest.mark.parametrize("config,n_inst,precision", [(3, None, tv.BF16), (4, None, tv.FP32), (5, 4, tv.BF16)])
def test_train_step_matches_separate_calls_other_graphs(config, n_inst, precision):
    # dense (SK), elimination (random regular) and mixed-size strip instances:
    # the one-call step against the separate entry points, one step
    w = wl.workload(config, n_inst) if n_inst else wl.workload(config)
    from paper_2504_12037_gb300.model import TNVAN

    n = len(w.graphs)
    B = 300
    mk = lambda: TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, seed=6)
    a, b = mk(), mk()
    dba = torch.empty(n * B, dtype=torch.float64, device="cuda")
    dja = torch.empty(sum(a.n_edges), dtype=torch.float64, device="cuda")
    dbb, djb = torch.empty_like(dba), torch.empty_like(dja)
    outa, outb = a.buffers(B), b.buffers(B)
    a.train_step(B, 5, 0, precision, 0.01, outa, dba, dja)
    b.train_step_separate(B, 5, 0, precision, 0.01, outb, dbb, djb)
    torch.cuda.synchronize()
    for x, y in zip(outa, outb):
        assert torch.equal(x, y)
    assert torch.equal(dba, dbb)
    assert torch.allclose(dja, djb, rtol=1e-12, atol=1e-12)
    assert torch.equal(a.grad, b.grad)
    assert torch.allclose(a.params, b.params, rtol=1e-6, atol=1e-9)
