"""The backward forms of Eq. 10 in the reduced-precision modes, against the
oracle's REINFORCE gradient on the same samples: for networks the fused BF16
kernel does not take, the tensor-core GEMM chain or the FP32 SIMT backward the
autotuner may pick instead, and the fused kernel on a width set of 83 spins
(padded to 96); and a multi-instance call mixing instances the fused kernel
takes (width sets padded to a multiple of 16) with others."""
import numpy as np
import pytest
import torch

from oracle import estimators as est
from oracle import made
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import oracle_samples, to_dev_spins

pytestmark = pytest.mark.gpu


def _case(w, n_inst, form, batch=200, seed=3):
    from paper_2504_12037_gb300.model import TNVAN

    model = TNVAN(w.graphs[:n_inst], w.widths_sets[:n_inst], w.hidden, w.betas[:n_inst], seed=seed, init_scale=1.5)
    model.ctx.set_tuning((0, 0, 0, 0, 0, 0, form))
    s_all, lq_all, lz_all, ref = [], [], [], []
    rng = np.random.default_rng(n_inst)
    for k in range(model.n):
        D = model.D[k]
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, D, w.hidden, 7, 1, k, batch)
        lq = made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, w.hidden, s_or).float().double()
        lz = torch.as_tensor(rng.normal(-50.0, 3.0, size=batch))  # any log Z_R: the gradient is linear in it
        ref.append(est.surrogate_grad(p32.astype(np.float64), D, w.hidden, s_or,
                                      est.reinforce_weights(lz, lq, w.betas[k])))
        s_all.append(s_or.numpy().reshape(-1))
        lq_all.append(lq.numpy())
        lz_all.append(lz.numpy())
    d_spins = to_dev_spins(np.concatenate(s_all))
    logq = torch.as_tensor(np.concatenate(lq_all), dtype=torch.float32).cuda()
    logZR = torch.as_tensor(np.concatenate(lz_all)).cuda()
    grad = torch.full_like(model.params, float("nan"))
    model.ctx.profile(True)
    model.ctx.backward(model.betas, batch, d_spins, logZR, logq, tv.BF16, grad)
    torch.cuda.synchronize()
    ran = model.ctx.profile_read()
    model.ctx.profile(False)
    return model, grad, ref, ran


def _check(gk, ref, exact):
    assert torch.isfinite(gk).all()
    if exact:  # FP32 arithmetic
        assert float((gk - ref).abs().max()) <= 2e-5 * float(ref.abs().max())
    else:  # BF16 operands: relative Frobenius error and direction
        fro = float((gk - ref).norm() / ref.norm())
        cos = float(torch.nn.functional.cosine_similarity(gk, ref, dim=0))
        assert fro <= 1e-1 and cos >= 0.99, (fro, cos)


@pytest.mark.parametrize("cfg,form", [(1, 1), (1, 2), (3, 1), (3, 2), (4, 1), (4, 2)])
def test_backward_forms_match_oracle(cfg, form):
    w = wl.workload(cfg)
    model, grad, ref, ran = _case(w, len(w.graphs), form)
    # the fused kernel takes workload 4 only (D = 83 with 2 x 128 units: 128 +
    # 96 + 144 + 144 TMEM columns with the layer-1 ones column in the padding,
    # 213 KB of shared memory with dX and dA2 in one buffer); workloads 1 (one
    # hidden layer) and 3 (256-unit layers) take the chosen form
    fused = cfg == 4
    assert model.ctx.instance_info(0)["fused_bwd"] == int(fused)
    assert ("bwd_fused" in ran) == fused
    assert ("backward" in ran) == (form == 2 and not fused)
    assert ("gemm_wgrad" in ran) == (form == 1 and not fused)
    for k in range(model.n):
        _check(grad[model.offsets[k]:model.offsets[k + 1]].cpu().double(), ref[k], form == 2 and not fused)


@pytest.mark.parametrize("form", [1, 2])
def test_mixed_fused_and_unfused_instances(form):
    # ten of the multi-instance workload's lattices (width sets of 16, 36, 64,
    # 144 and 256 spins): instances whose padded width set fits the fused
    # kernel's TMEM (D <= 80 with two hidden layers of 128) take it, the others
    # the chosen form, in one call; every instance's gradient against the oracle
    w = wl.workload(5, n_instances=10)
    model, grad, ref, ran = _case(w, 10, form, batch=160)
    # fused: the width sets of 16, 36 and 64 spins (36: the layer-1 ones column
    # sits in the padding, column 36 of 48)
    fused = [model.ctx.instance_info(k)["fused_bwd"] == 1 for k in range(model.n)]
    assert fused == [d <= 64 for d in model.D]
    assert any(fused) and not all(fused)
    assert any(f and d % 16 for f, d in zip(fused, model.D))
    assert "bwd_fused" in ran and (("backward" in ran) == (form == 2)) and (("gemm_wgrad" in ran) == (form == 1))
    for k in range(model.n):
        _check(grad[model.offsets[k]:model.offsets[k + 1]].cpu().double(), ref[k], form == 2 and not fused[k])
        if fused[k]:  # the layer-1 bias gradient (the ones column of [S | 1]) on its own
            H1, D = w.hidden[0], model.D[k]
            o = model.offsets[k] + H1 * D
            _check(grad[o:o + H1].cpu().double(), ref[k][H1 * D:H1 * D + H1], False)


@pytest.mark.parametrize("hidden", [[64, 128], [128, 64]])
def test_fused_backward_unequal_hidden_widths(hidden):
    # the fused kernel's three weight-gradient accumulators with H1 != H2
    # (TMEM 128 + 80 + (H1 + 16) + (H2 + 16) columns), against the oracle
    g = wl.lattice(16, 16, "gauss", seed=91)
    W = wl.width_columns(16, 16, wl.every_kth_column(16))
    w = wl.Workload("unequal", [g, g], [W, W], hidden, 200, [0.6, 1.0])
    model, grad, ref, ran = _case(w, 2, 0, batch=200)
    assert model.ctx.instance_info(0)["fused_bwd"] == 1
    assert "bwd_fused" in ran
    for k in range(model.n):
        _check(grad[model.offsets[k]:model.offsets[k + 1]].cpu().double(), ref[k], False)
