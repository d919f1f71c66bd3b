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
