"""The BF16 tensor-core sampler (tcgen05, Eq. 6-8) on every workload: one or
two hidden layers, hidden widths 16 to 256, width sets of 4 to 256 spins
(padded to a multiple of 16), mixed instance sizes in one launch.  log q is
checked against the FP64 oracle (teacher-forced on oracle-drawn samples, and on
the GPU's own samples), the sampler against its own teacher-forced log q, and
the distribution of a small network against its exact marginal."""
import numpy as np
import pytest
import torch

from oracle import ising, made
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import oracle_samples, to_dev_spins

pytestmark = pytest.mark.gpu

TOL_RED = 1e-3  # |delta log q| / N in the reduced-precision modes


def _model(w, n_inst=None, seed=3, scale=1.5):
    from paper_2504_12037_gb300.model import TNVAN

    n = len(w.graphs) if n_inst is None else n_inst
    return TNVAN(w.graphs[:n], w.widths_sets[:n], w.hidden, w.betas[:n], seed=seed, init_scale=scale)


def _workload(cfg):
    return wl.workload(cfg, n_instances=10) if cfg == 5 else wl.workload(cfg)


# plan values: the grouped form (4, 6, 8 steps per group; two hidden layers
# of <= 256 units, D <= 256 padded to 16: workloads 2, 3, 4 and 5, with
# weights streamed per group for workload 3's 256-unit layers and workload 5's
# D = 144 and 256) and the per-step form (12, 16, 32 steps per chunk; every
# shape)
@pytest.mark.parametrize("cfg,chunk", [(c, v) for c in (1, 2, 3, 4, 5) for v in (12, 16, 32)] +
                         [(c, v) for c in (2, 3, 4, 5) for v in (4, 6, 8)])
def test_tc_log_prob_matches_oracle_every_workload(cfg, chunk):
    w = _workload(cfg)
    model = _model(w)
    model.ctx.set_tuning((0, 0, 0, 0, chunk, 0))
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
    worst = 0.0
    for k in range(model.n):
        err = float((logq[k * batch:(k + 1) * batch].cpu().double() - refs[k]).abs().max()) / w.graphs[k].n
        worst = max(worst, err)
        assert err <= TOL_RED, (k, err)
    print(f"workload {cfg} chunk {chunk}: max |delta log q| / N = {worst:.2e}")


@pytest.mark.parametrize("cfg,plan", [(1, 0), (2, 0), (2, 16), (3, 0), (4, 0), (5, 0)])
def test_tc_sampler_own_samples_against_oracle(cfg, plan):
    # sampling on the tensor cores: log q of the GPU's own draws against the
    # oracle, and against the same kernel teacher-forced on those draws
    w = _workload(cfg)
    model = _model(w)
    model.ctx.set_tuning((0, 0, 0, 0, plan, 0))
    B = 300
    model.ctx.profile(True)
    spins, logq, _ = model.sample(B, 77, 5, precision=tv.BF16)
    torch.cuda.synchronize()
    assert "sample_tc" in model.ctx.profile_read()
    model.ctx.profile(False)
    lq2 = torch.empty_like(logq)
    model.ctx.log_prob(B, spins, lq2, tv.BF16)
    torch.cuda.synchronize()
    assert torch.allclose(logq, lq2, atol=1e-5, rtol=0)
    for k in range(model.n):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy().astype(np.float64)
        s = torch.as_tensor(model.spins_of(spins, k, B).cpu().numpy().astype(np.float64))
        assert torch.all(s.abs() == 1)
        ref = made.log_q(torch.as_tensor(p32), model.D[k], w.hidden, s)
        err = float((logq[k * B:(k + 1) * B].cpu().double() - ref).abs().max()) / w.graphs[k].n
        assert err <= TOL_RED, (k, err)


def test_tc_sampler_one_hidden_layer_distribution():
    # the 4x4 workload's network (4 -> 16 -> 4, one hidden layer): the
    # frequencies of the 16 width-set states against the network's exact q
    w = wl.workload(1)
    model = _model(w, scale=2.0)
    B = 200000
    spins, logq, _ = model.sample(B, 4321, 0, precision=tv.BF16)
    s = model.spins_of(spins, 0, B).cpu().numpy()
    idx = (((1 - s) // 2) * (2 ** np.arange(4))).sum(1)
    counts = np.bincount(idx, minlength=16).astype(float)
    th = torch.as_tensor(model.params.cpu().numpy().astype(np.float64))
    q = torch.exp(made.log_q(th, 4, w.hidden, ising.all_configs(4))).numpy()
    chi2 = float(((counts - B * q) ** 2 / (B * q)).sum())
    print("chi2 (15 dof):", chi2)
    assert chi2 < 45


# grouped-form networks by in-group form (MADE hidden degrees k mod (D-1) + 1):
# 2 slots (D = 64, H = 64), 3 (workload 2's 64-128-128), 4 (D = 32, H = 96;
# D = 21, H = 64), the per-unit form (D = 16, H = 128: up to 9 units per
# degree), and weights streamed per step group (D = 144 and D = 256, H = 128)
GROUPED_SHAPES = [(16, 16, [64, 64], 2, 0), (16, 16, [128, 128], 3, 0), (16, 8, [96, 96], 4, 0),
                  (8, 8, [128, 128], 0, 0), (14, 7, [64, 64], 4, 0),  # D = 21, padded to 32
                  (24, 24, [128, 128], 2, 1), (32, 32, [128, 128], 2, 1),
                  # unequal hidden widths (slot count not pinned), resident and streamed
                  (16, 16, [64, 128], None, 0), (24, 24, [128, 64], None, 1)]


@pytest.mark.parametrize("plan", [4, 6, 8])
@pytest.mark.parametrize("shape", range(len(GROUPED_SHAPES)))
def test_tc_grouped_forms_against_oracle(shape, plan):
    from paper_2504_12037_gb300.model import TNVAN

    Lx, Ly, hidden, slots, streamed = GROUPED_SHAPES[shape]
    g = wl.lattice(Lx, Ly, "gauss", seed=31 + shape)
    W = wl.width_columns(Lx, Ly, wl.every_kth_column(Lx))
    model = TNVAN([g, g], [W, W], hidden, [0.6, 1.1], seed=4 + shape, init_scale=1.5)
    info = model.ctx.instance_info(0)
    assert (slots is None or info["tcg_slots"] == slots) and info["tcg_streamed"] == streamed, info
    model.ctx.set_tuning((0, 0, 0, 0, plan, 0))
    D, B = len(W), 300  # three CTAs, the last one ragged
    # teacher-forced on oracle draws
    s_all, refs = [], []
    for k in range(2):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_or, _, _ = oracle_samples(p32, D, hidden, 3, 0, k, B)
        s_all.append(s_or.numpy().reshape(-1))
        refs.append(made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, hidden, s_or))
    logq = torch.empty(2 * B, dtype=torch.float32, device="cuda")
    model.ctx.profile(True)
    model.ctx.log_prob(B, to_dev_spins(np.concatenate(s_all)), logq, tv.BF16)
    torch.cuda.synchronize()
    assert "log_prob_tc" in model.ctx.profile_read()
    for k in range(2):
        err = float((logq[k * B:(k + 1) * B].cpu().double() - refs[k]).abs().max()) / g.n
        assert err <= TOL_RED, (k, err)
    # own draws: log q against the oracle and the teacher-forced kernel; the
    # draws themselves against the oracle's replay of the same uniforms (rows
    # differ only where a BF16 probability falls on the other side of u)
    spins, lq_s, _ = model.sample(B, 77, 5, precision=tv.BF16)
    torch.cuda.synchronize()
    assert "sample_tc" in model.ctx.profile_read()
    model.ctx.profile(False)
    lq2 = torch.empty_like(lq_s)
    model.ctx.log_prob(B, spins, lq2, tv.BF16)
    torch.cuda.synchronize()
    assert torch.allclose(lq_s, lq2, atol=1e-5, rtol=0)
    for k in range(2):
        p32 = model.params[model.offsets[k]:model.offsets[k + 1]].cpu().numpy()
        s_gpu = model.spins_of(spins, k, B).cpu().numpy().astype(np.float64)
        ref = made.log_q(torch.as_tensor(p32, dtype=torch.float64), D, hidden, torch.as_tensor(s_gpu))
        err = float((lq_s[k * B:(k + 1) * B].cpu().double() - ref).abs().max()) / g.n
        assert err <= TOL_RED, (k, err)
        s_or, _, _ = oracle_samples(p32, D, hidden, 77, 5, k, B)
        same = np.all(s_gpu == s_or.numpy(), axis=1).mean()
        assert same >= 0.8, (k, same)
