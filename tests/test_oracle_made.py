"""Pins for oracle.made and oracle.philox (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import ising, made, philox


@pytest.mark.parametrize("D,H", [(6, [10, 10]), (5, []), (4, [16]), (7, [5, 9]), (1, [3])])
def test_normalised(D, H):
    th = torch.as_tensor(made.init_params(D, H, 1)) * 3
    assert abs(float(torch.exp(made.all_log_q(th, D, H)).sum()) - 1) < 1e-12


def test_zero_params_uniform():
    D, H = 8, [12, 12]
    th = torch.zeros(made.n_params(D, H), dtype=torch.float64)
    s = torch.tensor(np.random.default_rng(0).choice([-1.0, 1.0], size=(5, D)))
    assert torch.allclose(made.log_q(th, D, H, s), torch.full((5,), -D * math.log(2), dtype=torch.float64))


@pytest.mark.parametrize("D,H", [(6, [10, 10]), (5, []), (9, [20])])
def test_autoregressive_dependencies(D, H):
    # x_i must not depend on s_j for j >= i, and (generic weights) must depend on s_{i-1}.
    th = torch.as_tensor(made.init_params(D, H, 2)) * 4
    rng = np.random.default_rng(5)
    s = torch.tensor(rng.choice([-1.0, 1.0], size=(64, D)))
    x = made.logits(th, D, H, s)
    for j in range(D):
        s2 = s.clone()
        s2[:, j] = -s2[:, j]
        d = (made.logits(th, D, H, s2) - x).abs().max(0).values
        assert torch.all(d[: j + 1] == 0)
        if j + 1 < D:
            assert d[j + 1] > 0


def test_mask_counts_match_degree_rule():
    D, H = 5, [8]
    m = made.masks(D, H)
    deg_h = np.arange(8) % 4 + 1
    assert int(m[0].sum()) == sum(int(d) for d in deg_h)  # unit of degree d sees inputs 1..d
    assert int(m[1].sum()) == sum(int((np.arange(1, 6) > d).sum()) for d in deg_h)


def test_philox_known_answers():
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for c, k, out in cases:
        got = philox.philox4x32_10(np.array(c, np.uint64), np.array(k, np.uint64))
        assert [int(x) for x in got] == out


def test_uniforms_layout_and_range():
    u = philox.uniforms(7, 3, 2, 10, 9)
    assert u.shape == (10, 9) and u.min() >= 0 and u.max() < 1
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))
    # spin i uses word i & 3 of counter block i >> 2
    w = philox.philox4x32_10(np.array([4, 1, 3, 2], np.uint64), np.array([7, 0], np.uint64))
    assert u[4, 6] == float(int(w[2]) >> 8) * 2.0 ** -24


def test_sampler_distribution_matches_q():
    D, H = 4, [16]
    th = torch.as_tensor(made.init_params(D, H, 9)) * 3
    B = 200000
    u = philox.uniforms(11, 0, 0, B, D)
    s, p = made.sample(th, D, H, u)
    idx = (((1 - s) / 2).long() * (2 ** torch.arange(D))).sum(1)
    counts = torch.bincount(idx, minlength=2 ** D).double()
    q = torch.exp(made.all_log_q(th, D, H))
    chi2 = float(((counts - B * q) ** 2 / (B * q)).sum())
    assert chi2 < 45  # 15 dof, p ~ 1e-4
    # the sampler's own conditionals reproduce log q
    lq = made.log_q(th, D, H, s[:1000])
    lp = torch.where(s[:1000] > 0, torch.log(p[:1000]), torch.log1p(-p[:1000])).sum(1)
    assert torch.allclose(lq, lp, atol=1e-12)


def test_sampler_threshold_convention():
    D, H = 3, [4]
    th = torch.zeros(made.n_params(D, H), dtype=torch.float64)
    u = np.array([[0.5 - 2 ** -24, 0.5, 0.0]])
    s, _ = made.sample(th, D, H, u)
    assert s.tolist() == [[1.0, -1.0, 1.0]]  # s = +1 iff u < p (strict)
