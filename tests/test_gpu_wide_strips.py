"""GPU parity of the wide-strip contraction (lattice width sets leaving strips
of 5 to 12 columns: every state-count class of the kernel) against the FP64
oracle's exact elimination, through the C-ABI, and against the GPU's own
elimination plan of the same instances (the path taken when d/dbeta is
requested).  Width-set rows are seeded inputs."""
import numpy as np
import pytest
import torch

from oracle import general
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

from gpu_helpers import to_dev_spins

pytestmark = pytest.mark.gpu

# (Lx, Ly, W columns, couplings): strip widths 5, 6, 6 | 7, 8, 12 | 9, 10, 5 | 11, 1
CASES = [
    (20, 10, [5, 12, 19], "gauss"),
    (30, 8, [7, 16, 29], "gauss"),
    (26, 9, [9, 20], "pm1"),
    (13, 12, [11], "ferro"),
]


def _instances(cases):
    gs, Ws = [], []
    for i, (Lx, Ly, cols, dist) in enumerate(cases):
        gs.append(wl.lattice(Lx, Ly, dist, seed=70 + i))
        Ws.append(wl.width_columns(Lx, Ly, cols))
    return gs, Ws


def test_wide_strips_match_oracle_and_elimination():
    from paper_2504_12037_gb300.model import TNVAN

    gs, Ws = _instances(CASES)
    betas = [0.8, 1.1, 0.6, 1.0 / 2.269185]
    model = TNVAN(gs, Ws, [32, 32], betas, seed=3)
    for k in range(len(gs)):
        assert model.ctx.instance_info(k)["kind"] == 2  # elimination plan (with the wide-strip forward)
    B = 150  # ragged against everything
    rng = np.random.default_rng(12)
    s_all = [np.where(rng.random((B, len(W))) < 0.5, 1.0, -1.0) for W in Ws]
    d_spins = to_dev_spins(np.concatenate([s.reshape(-1) for s in s_all]))
    n = len(gs)
    lz_wide = torch.empty(n * B, dtype=torch.float64, device="cuda")
    model.ctx.profile(True)
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, lz_wide)
    torch.cuda.synchronize()
    ran = model.ctx.profile_read()
    model.ctx.profile(False)
    assert "wide_strips" in ran and "general" not in ran
    # the elimination plan of the same instances (d/dbeta requested)
    lz_el = torch.empty_like(lz_wide)
    db = torch.empty_like(lz_wide)
    model.ctx.contract(model.betas, B, d_spins, tv.FP32, lz_el, db)
    torch.cuda.synchronize()
    lw, le = lz_wide.cpu().numpy(), lz_el.cpu().numpy()
    rows = np.arange(0, B, 7)
    for k, (g, W) in enumerate(zip(gs, Ws)):
        sl = slice(k * B, (k + 1) * B)
        assert np.abs(lw[sl] - le[sl]).max() / g.n <= 1e-6, k
        ref = general.log_zr_general(g.n, g.ei, g.ej, g.J, betas[k], W, torch.as_tensor(s_all[k][rows]),
                                     enum_max=0).numpy()
        err = np.abs(lw[sl][rows] - ref).max() / g.n
        print(f"instance {k}: max |delta log Z_R| / N = {err:.2e}")
        assert err <= 1e-6, (k, err)


def test_wide_strips_beside_other_kinds_and_in_training_step():
    # a wide-strip lattice beside a narrow-strip lattice and a dense block in
    # one context: each kind contracts its own instances
    from paper_2504_12037_gb300.model import TNVAN

    g1 = wl.lattice(20, 10, "gauss", seed=81)
    W1 = wl.width_columns(20, 10, [6, 13])
    g2 = wl.lattice(8, 8, "gauss", seed=82)
    W2 = wl.width_columns(8, 8, wl.every_kth_column(8))
    g3 = wl.sk(20, 83)
    W3 = np.arange(6, dtype=np.int32)
    gs, Ws, betas = [g1, g2, g3], [W1, W2, W3], [0.9, 0.9, 0.9]
    model = TNVAN(gs, Ws, [32, 32], betas, seed=4)
    B = 96
    spins, logq, logZR = model.sample(B, 5, 1, tv.FP32)
    torch.cuda.synchronize()
    lz = logZR.cpu().numpy()
    for k, (g, W) in enumerate(zip(gs, Ws)):
        s = model.spins_of(spins, k, B).cpu().numpy().astype(np.float64)[::5]
        ref = general.log_zr_general(g.n, g.ei, g.ej, g.J, betas[k], W, torch.as_tensor(s), enum_max=0).numpy()
        assert np.abs(lz[k * B:(k + 1) * B][::5] - ref).max() / g.n <= 1e-6, k
    # a training step runs through the same contraction
    bufs = model.buffers(B)
    model.train_step(B, 5, 2, tv.FP32, 0.01, bufs, None, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.isfinite(bufs[2]).all()
