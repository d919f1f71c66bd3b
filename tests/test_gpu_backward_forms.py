"""The two backward forms of networks the fused BF16 kernel does not take
(Eq. 10): the tensor-core GEMM chain (BF16 operands) and the FP32 SIMT
backward the autotuner may pick in its place in the reduced-precision modes,
against the oracle's REINFORCE gradient on the same samples."""
import numpy as np
import pytest
import torch

from oracle import estimators as est
from oracle import made
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import oracle_samples, to_dev_spins

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,form", [(4, 1), (4, 2), (1, 2), (3, 2)])
def test_backward_forms_match_oracle(cfg, form):
    from paper_2504_12037_gb300.model import TNVAN

    w = wl.workload(cfg)
    model = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, seed=3, init_scale=1.5)
    model.ctx.set_tuning((0, 0, 0, 0, 0, 0, form))
    batch = 200
    s_all, lq_all, lz_all, ref = [], [], [], []
    rng = np.random.default_rng(cfg)
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
    assert ("backward" in ran) == (form == 2) and ("gemm_wgrad" in ran) == (form == 1)
    for k in range(model.n):
        gk = grad[model.offsets[k]:model.offsets[k + 1]].cpu().double()
        if form == 2:  # FP32 arithmetic
            assert float((gk - ref[k]).abs().max()) <= 2e-5 * float(ref[k].abs().max())
        else:
            fro = float((gk - ref[k]).norm() / ref[k].norm())
            cos = float(torch.nn.functional.cosine_similarity(gk, ref[k], dim=0))
            assert fro <= 1e-1 and cos >= 0.99
