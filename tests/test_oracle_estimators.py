"""Pins for oracle.estimators: Jensen, Eq. 5, finite differences, Adam."""
import math

import numpy as np
import pytest
import torch

from oracle import estimators as est
from oracle import ising, made, philox
from paper_2504_12037_gb300 import workloads as wl


def _cfg1():
    w = wl.workload(1)
    g, W = w.graphs[0], w.widths_sets[0]
    lzr_all = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 1.0, W, ising.all_configs(len(W)))
    return g, W, lzr_all


def test_is_below_fq_every_batch():
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.standard_normal(50) * 3, rng.standard_normal(50)
        r = est.free_energies(a, b, 0.7)
        assert r["F_IS"] <= r["F_q"] + 1e-15


def test_uniform_q_exact_fq_closed_form():
    g, W, lzr = _cfg1()
    D = len(W)
    th = torch.zeros(made.n_params(D, [16]), dtype=torch.float64)
    fq = float(est.exact_fq(th, D, [16], lzr, 1.0))
    assert abs(fq - (-(float(lzr.mean()) + D * math.log(2)))) < 1e-12


def test_exact_fq_upper_bounds_f():
    g, W, lzr = _cfg1()
    F = -float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, 1.0))
    for seed in range(5):
        th = torch.as_tensor(made.init_params(len(W), [16], seed)) * 2
        assert float(est.exact_fq(th, len(W), [16], lzr, 1.0)) >= F - 1e-12


def test_exact_fq_reaches_f_when_q_is_p():
    # With no hidden layer and D = 1 the network's bias alone can equal p exactly.
    g = wl.lattice(3, 3, "gauss", 4)
    W = np.array([4], np.int32)
    lzr = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 0.9, W, ising.all_configs(1))
    p_up = torch.softmax(lzr, 0)[0]
    th = torch.tensor([0.0, float(torch.log(p_up / (1 - p_up)))], dtype=torch.float64)
    F = -float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, 0.9)) / 0.9
    assert abs(float(est.exact_fq(th, 1, [], lzr, 0.9)) - F) < 1e-12


def test_surrogate_gradient_finite_differences():
    D, H = 5, [7, 6]
    th = made.init_params(D, H, 3) * 2
    s = torch.tensor(np.random.default_rng(1).choice([-1.0, 1.0], size=(40, D)))
    w = torch.tensor(np.random.default_rng(2).standard_normal(40))
    g = est.surrogate_grad(th, D, H, s, w)
    f = lambda t: float((w * made.log_q(torch.as_tensor(t), D, H, s)).sum())
    for k in np.random.default_rng(3).choice(th.size, 25, replace=False):
        e = np.zeros_like(th)
        e[k] = 1e-6
        fd = (f(th + e) - f(th - e)) / 2e-6
        assert abs(fd - float(g[k])) < 1e-7 * max(1, abs(fd))


def test_exact_gradient_finite_differences():
    g_, W, lzr = _cfg1()
    D, H = len(W), [16]
    th = made.init_params(D, H, 4)
    g = est.exact_grad(th, D, H, lzr, 1.0)
    for k in range(0, th.size, 7):
        e = np.zeros_like(th)
        e[k] = 1e-6
        fd = (float(est.exact_fq(th + e, D, H, lzr, 1.0)) - float(est.exact_fq(th - e, D, H, lzr, 1.0))) / 2e-6
        assert abs(fd - float(g[k])) < 1e-7


def test_sampled_reinforce_gradient_is_unbiased():
    g_, W, lzr = _cfg1()
    D, H = len(W), [16]
    th = made.init_params(D, H, 4)
    exact = est.exact_grad(th, D, H, lzr, 1.0)
    reps = []
    for rep in range(40):
        u = philox.uniforms(99, rep, 0, 512, D)
        s, _ = made.sample(torch.as_tensor(th), D, H, u)
        idx = (((1 - s) / 2).long() * (2 ** torch.arange(D))).sum(1)
        lq = made.log_q(torch.as_tensor(th), D, H, s)
        w = est.reinforce_weights(lzr[idx], lq, 1.0)
        reps.append(est.surrogate_grad(th, D, H, s, w))
    G = torch.stack(reps)
    mean, se = G.mean(0), G.std(0) / math.sqrt(G.shape[0])
    z = ((mean - exact).abs() / (se + 1e-12))
    assert float((z < 4.5).double().mean()) > 0.97


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = est.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, -0.01 * np.sign(g), atol=1e-15)


def test_is_energy_over_all_width_states_is_the_exact_internal_energy():
    # every width-set state once with the uniform log q = -D ln 2: the weights
    # are Z_R(s) / sum Z_R = the exact marginal of s, so sum_s w_s E_s with
    # E_s = -d log Z_R(s) / d beta is the exact <E> = -d log Z / d beta
    g, W, _ = _cfg1()
    D = len(W)
    for beta in (0.4, 1.0, 1.7):
        bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        lzr = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, bt, W, ising.all_configs(D))
        E = -torch.stack([torch.autograd.grad(lzr[i], bt, retain_graph=True)[0] for i in range(lzr.shape[0])])
        U, Uq, ess = est.is_observables(lzr.detach(), torch.full((lzr.shape[0],), -D * math.log(2.0)), E)
        b2 = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        (dlz,) = torch.autograd.grad(ising.log_z_brute(g.n, g.ei, g.ej, g.J, b2), b2)
        assert abs(U - (-float(dlz))) < 1e-10 * max(1.0, abs(U))
        assert 1.0 <= ess <= lzr.shape[0]
        # the conditional energy is the Boltzmann mean of E(s, r) over r given s (brute force)
        s0 = ising.all_configs(D)[3:4]
        n_r = g.n - D
        R = [v for v in range(g.n) if v not in set(int(x) for x in W)]
        full = torch.empty((1 << n_r, g.n), dtype=torch.float64)
        full[:, W] = s0
        full[:, R] = ising.all_configs(n_r)
        en = ising.energy(g.ei, g.ej, g.J, full)
        p = torch.softmax(-beta * en, 0)
        assert abs(float((p * en).sum()) - float(E[3])) < 1e-10 * max(1.0, abs(float(E[3])))


def test_is_uniform_weights():
    lz = torch.linspace(-3.0, 2.0, 7, dtype=torch.float64)
    U, Uq, ess = est.is_observables(lz, lz, torch.arange(7, dtype=torch.float64))
    assert abs(U - Uq) < 1e-12 and abs(ess - 7.0) < 1e-12


# --- free_energies: the -ln B of log Z_IS, the ddof of the stderr, the mean ---

def test_constant_l_gives_equal_free_energies_and_zero_stderr():
    # l_b = c for every sample: mean = c and logsumexp - ln B = c + ln B - ln B,
    # so F_q = F_IS = -c / beta whatever B is; a dropped (or doubled) ln B moves
    # F_IS by ln B / beta.  The spread is zero.
    for B in (1, 2, 7, 1000):
        for c, beta in ((-3.25, 0.5), (41.0, 2.0)):
            lz = np.full(B, c + 1.5)
            lq = np.full(B, 1.5)
            r = est.free_energies(lz, lq, beta)
            assert abs(r["F_q"] - (-c / beta)) < 1e-12
            assert abs(r["F_IS"] - (-c / beta)) < 1e-12
            assert abs(r["logZ_IS"] - c) < 1e-12
            assert r["stderr"] == 0.0


def test_three_sample_hand_values():
    # l = (0, ln 2, ln 6): the mean importance weight is (1 + 2 + 6) / 3 = 3,
    # so log Z_IS = ln 3; the mean of l is ln 12 / 3.
    l = np.array([0.0, math.log(2.0), math.log(6.0)])
    r = est.free_energies(l, np.zeros(3), 0.5)
    assert abs(r["logZ_IS"] - math.log(3.0)) < 1e-14
    assert abs(r["F_IS"] - (-2.0 * math.log(3.0))) < 1e-14
    assert abs(r["F_q"] - (-2.0 * math.log(12.0) / 3.0)) < 1e-14
    # l = (1, 2, 6), beta = 2: mean 3, squared deviations 4 + 1 + 9 = 14, so the
    # unbiased variance (ddof 1) is 7 and stderr = sqrt(7) / (2 sqrt(3)); the
    # biased form would give sqrt(14/3) / (2 sqrt(3)).
    r = est.free_energies(np.array([1.0, 2.0, 6.0]), np.zeros(3), 2.0)
    assert abs(r["F_q"] - (-1.5)) < 1e-14
    assert abs(r["stderr"] - math.sqrt(7.0) / (2.0 * math.sqrt(3.0))) < 1e-14


def test_is_estimate_is_exact_for_exact_q_and_for_a_full_uniform_census():
    # Eq. 5 / Eq. 9: if q(s) equals the Boltzmann marginal p(s) = Z_R(s) / Z of
    # the width set, every l_b = log Z_R(s_b) - log p(s_b) = ln Z, so F_q = F_IS
    # = F (brute force) on any samples and the stderr vanishes.
    g, W, lzr = _cfg1()
    D = len(W)
    logZ = float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, 1.0))
    F = -logZ
    log_p = lzr - torch.logsumexp(lzr, 0)
    idx = np.random.default_rng(5).integers(0, 2 ** D, size=333)
    r = est.free_energies(lzr[idx], log_p[idx], 1.0)
    assert abs(r["F_q"] - F) < 1e-12 and abs(r["F_IS"] - F) < 1e-12
    assert r["stderr"] < 1e-12
    # Uniform q (log q = -D ln 2) over every width-set state once, B = 2^D:
    # logsumexp(l) = ln sum_s Z_R(s) + D ln 2 = ln Z + ln B (Eq. 3), so F_IS = F
    # exactly while F_q >= F (Jensen).
    r = est.free_energies(lzr, torch.full_like(lzr, -D * math.log(2.0)), 1.0)
    assert abs(r["F_IS"] - F) < 1e-12
    assert r["F_q"] > F


def test_is_estimate_converges_on_uniform_samples():
    # B = 2^15 uniform draws of the 16 width states of the 4x4 workload: F_IS
    # approaches the brute-force F; the gap is far below the per-sample spread
    g, W, lzr = _cfg1()
    D = len(W)
    F = -float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, 1.0))
    idx = np.random.default_rng(8).integers(0, 2 ** D, size=1 << 15)
    r = est.free_energies(lzr[idx], torch.full((idx.size,), -D * math.log(2.0), dtype=torch.float64), 1.0)
    assert abs(r["F_IS"] - F) < 4.0 * r["stderr"]
    assert r["F_IS"] <= r["F_q"]


# --- adam_step beyond the first step ---

def test_adam_constant_gradient_closed_form():
    # With g_t = g for every t: m_t = g (1 - b1^t) and v_t = g^2 (1 - b2^t), so
    # the bias-corrected moments are g and g^2 at every t and each update is
    # lr g / (|g| + eps): after t steps p = -t lr g / (|g| + eps).  eps = 0.1
    # makes the placement of eps (outside the square root) visible.
    g = np.array([0.5, -2.0, 3e-3])
    lr, eps = 0.05, 0.1
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        p, m, v = est.adam_step(p, g, m, v, t, lr=lr, eps=eps)
        assert np.allclose(p, -t * lr * g / (np.abs(g) + eps), rtol=1e-13, atol=0)


def test_adam_zero_then_g_closed_form():
    # g_1 = 0, g_2 = g: m_2 = (1 - b1) g, v_2 = (1 - b2) g^2; corrected by
    # 1 - b1^2 = (1 - b1)(1 + b1) and 1 - b2^2 = (1 - b2)(1 + b2) they are
    # g / (1 + b1) and g^2 / (1 + b2), so the second update is
    # lr (g / (1 + b1)) / (|g| / sqrt(1 + b2) + eps).
    b1, b2, lr, eps = 0.9, 0.999, 0.01, 0.05
    g = np.array([1.25, -0.4])
    p, m, v = est.adam_step(np.zeros(2), np.zeros(2), np.zeros(2), np.zeros(2), 1, lr=lr, b1=b1, b2=b2, eps=eps)
    assert np.all(p == 0.0)
    p, m, v = est.adam_step(p, g, m, v, 2, lr=lr, b1=b1, b2=b2, eps=eps)
    want = -lr * (g / (1 + b1)) / (np.abs(g) / math.sqrt(1 + b2) + eps)
    assert np.allclose(p, want, rtol=1e-13, atol=0)
