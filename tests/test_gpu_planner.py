"""GPU parity of elimination plans built by the width-set finder (Sec. 2):
random regular graphs with W and R's elimination order from
tnvan_find_width_set (larger components than the greedy width-set workload,
forward passes on the reused table layout), against the oracle's own
elimination in its min-degree order: log q, log Z_R and d/dbeta on oracle
samples, d/dJ by autograd, log Z_R on the GPU's own BF16 samples, and the
ordered width-set call's argument checks."""
import numpy as np
import pytest
import torch

from oracle import general
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl
from paper_2504_12037_gb300.model import TNVAN

from gpu_helpers import oracle_samples, to_dev_spins
from test_gpu_dense_general import _parity

pytestmark = pytest.mark.gpu
HIDDEN = [32]


def _planned(n, d, wu, seed):
    g = wl.random_regular(n, d, seed)
    W, order, width, _ = tv.find_width_set(g.n, g.ei, g.ej, wu, restarts=2, seed=1)
    return g, W, order, width


@pytest.mark.parametrize("n,d,wu", [(1000, 3, 8), (1000, 3, 2), (256, 3, 8), (300, 4, 5), (300, 3, 12)])
def test_planned_rrg_contraction_parity(n, d, wu):
    g, W, order, width = _planned(n, d, wu, 12037 + 6000 + n + d)
    model = TNVAN([g], [W], HIDDEN, [1.0], seed=5, init_scale=1.5, elim_orders=[order])
    info = model.ctx.instance_info(0)
    assert info["kind"] == 2 and info["max_width"] == width <= wu
    assert 0 < info["arena_live"] <= info["arena"]
    _parity(model, [g], [W], HIDDEN, [1.0], batch=40)


@pytest.mark.parametrize("n,wu", [(1000, 8), (300, 12)])
def test_planned_rrg_dJ_parity(n, wu):
    g, W, order, _ = _planned(n, 3, wu, 12037 + 6000 + n + 3)
    beta = 0.7
    model = TNVAN([g], [W], HIDDEN, [beta], seed=5, init_scale=1.5, elim_orders=[order])
    B = 20
    p32 = model.params.cpu().numpy()
    s_or, _, _ = oracle_samples(p32, len(W), HIDDEN, 3, 0, 0, B)
    Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lz = general.log_zr_general(g.n, g.ei, g.ej, Jt, beta, W, s_or)
    (ref,) = torch.autograd.grad(lz.mean(), Jt)
    d_spins = to_dev_spins(s_or.numpy().reshape(-1))
    logZR = torch.empty(B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, logZR)
    dJ = torch.empty(g.m, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(model.params)
    model.ctx.backward(model.betas, B, d_spins, logZR, torch.zeros(B, dtype=torch.float32, device="cuda"),
                       tv.FP32, grad, None, dJ)
    torch.cuda.synchronize()
    assert float((logZR.cpu() - lz.detach()).abs().max()) / g.n <= 1e-6
    assert float((dJ.cpu() - ref).abs().max()) <= 2e-5 * max(1.0, float(ref.abs().max()))


def test_planned_rrg_bf16_samples_and_free_energy():
    g, W, order, _ = _planned(1000, 3, 4, 12037 + 6000 + 1003)
    model = TNVAN([g], [W], [64, 64], [0.5], seed=2, elim_orders=[order])
    B = 4096
    spins, logq, logZR = model.sample(B, seed=7, step=1, precision=tv.BF16)
    fe = model.free_energy(B, logZR, logq)
    torch.cuda.synchronize()
    assert np.isfinite(fe).all() and fe[0, 1] <= fe[0, 0] + 1e-9  # F_IS <= F_q per batch
    rows = [0, 1, 777, B - 1]
    s = model.spins_of(spins, 0, B)[rows].cpu().to(torch.float64)
    ref = general.log_zr_general(g.n, g.ei, g.ej, g.J, 0.5, W, s)
    assert float((logZR[rows].cpu() - ref).abs().max()) / g.n <= 1e-3


def test_ordered_width_set_arguments():
    g, W, order, _ = _planned(256, 3, 8, 12037 + 6000 + 259)
    ctx = tv.Context(0)
    ctx.init_graph(0, g.n, g.ei, g.ej, g.J, g.topology)
    bad = order.copy()
    bad[0] = W[0]  # a W spin in R's order
    with pytest.raises(tv.TnvanError) as e:
        ctx.set_width_set(0, W, bad)
    assert e.value.code == tv.E_ARG
    with pytest.raises(tv.TnvanError) as e:
        ctx.set_width_set(0, W, np.concatenate([order[:-1], order[:1]]))  # a repeated spin
    assert e.value.code == tv.E_ARG
    ctx.set_width_set(0, W, order)
    assert ctx.instance_info(0)["max_width"] <= 8
    # an order whose width exceeds the kernels' limit (12) is refused
    W1, o1, w1, _ = tv.find_width_set(g.n, g.ei, g.ej, 16, restarts=1, seed=1)
    assert w1 > 12
    with pytest.raises(tv.TnvanError) as e:
        ctx.set_width_set(0, W1, o1)
    assert e.value.code == tv.E_UNSUPPORTED
    # lattice plans take no order
    lat = wl.lattice(8, 8, "gauss", seed=1)
    Wl = wl.width_columns(8, 8, [3])
    ctx.init_graph(1, lat.n, lat.ei, lat.ej, lat.J, lat.topology, lat.Lx, lat.Ly)
    Rl = np.array([v for v in range(lat.n) if v not in set(Wl.tolist())], np.int32)
    with pytest.raises(tv.TnvanError) as e:
        ctx.set_width_set(1, Wl, Rl)
    assert e.value.code == tv.E_ARG
    ctx.close()


def test_planned_rrg_full_size_sampled_rows():
    """The bench's planned workload at full size (n = 1000, d = 3, w_u = 8,
    batch 10,000, global tables, lane groups): log Z_R and d/dbeta on sampled
    rows against the oracle, and sum_e J_e dlogZ/dJ_e = beta dlogZ/dbeta over
    the whole batch (log Z_R depends on beta and J only through beta J)."""
    g = wl.random_regular(1000, 3, 12037 + 7000)
    W, order, _, _ = tv.find_width_set(g.n, g.ei, g.ej, 8, restarts=4, seed=1)
    beta = 0.5
    model = TNVAN([g], [W], [128, 128], [beta], seed=5, elim_orders=[order])
    B = 10000
    spins, logq, logZR = model.sample(B, seed=3, step=1, precision=tv.BF16)
    dbeta = torch.empty(B, dtype=torch.float64, device="cuda")
    model.ctx.contract(model.betas, B, spins, tv.FP32, logZR, dbeta)
    dJ = torch.empty(g.m, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(model.params)
    model.ctx.backward(model.betas, B, spins, logZR, logq, tv.FP32, grad, None, dJ)
    torch.cuda.synchronize()
    rows = [0, 1, 4321, 9998, B - 1]
    s = model.spins_of(spins, 0, B)[rows].cpu().to(torch.float64)
    bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    lz = general.log_zr_general(g.n, g.ei, g.ej, g.J, bt, W, s)
    db_ref = torch.stack([torch.autograd.grad(lz[i], bt, retain_graph=True)[0] for i in range(len(rows))])
    assert float((logZR[rows].cpu() - lz.detach()).abs().max()) / g.n <= 1e-6
    assert float((dbeta[rows].cpu() - db_ref).abs().max()) <= 2e-5 * max(1.0, float(db_ref.abs().max()))
    lhs = float((torch.as_tensor(g.J, dtype=torch.float64) * dJ.cpu()).sum())
    rhs = beta * float(dbeta.mean())
    assert abs(lhs - rhs) <= 1e-5 * max(1.0, abs(rhs))
