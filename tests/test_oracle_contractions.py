"""Pins for oracle.dense, oracle.general and the contraction derivatives."""
import math

import numpy as np
import pytest
import torch

from oracle import dense, general, ising, transfer
from paper_2504_12037_gb300 import workloads as wl


def test_dense_equals_enumeration_small_sk():
    g = wl.sk(14, 5)
    W = np.arange(9, dtype=np.int32)
    sW = torch.tensor(np.random.default_rng(0).choice([-1.0, 1.0], size=(7, 9)))
    for beta in (0.5, 2.0):
        a = dense.log_zr_dense(g.n, g.ei, g.ej, g.J, beta, W, sW)
        b = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, beta, W, sW)
        assert torch.allclose(a, b, atol=1e-12, rtol=0)


def test_dense_factorisation_equals_brute_force():
    g = wl.sk(12, 6)
    W = np.array([0, 3, 5, 6, 8, 9, 10, 11], np.int32)
    lzr = dense.log_zr_dense(g.n, g.ei, g.ej, g.J, 1.3, W, ising.all_configs(8))
    ref = float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, 1.3))
    assert abs(float(torch.logsumexp(lzr, 0)) - ref) < 1e-12 * abs(ref)


def test_general_enumeration_and_elimination_match():
    g = wl.random_regular(20, 3, 7)
    W = np.array([0, 5, 9, 13], np.int32)
    sW = torch.tensor(np.random.default_rng(1).choice([-1.0, 1.0], size=(5, 4)))
    ref = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 1.0, W, sW)
    a = general.log_zr_general(g.n, g.ei, g.ej, g.J, 1.0, W, sW, enum_max=16)
    b = general.log_zr_general(g.n, g.ei, g.ej, g.J, 1.0, W, sW, enum_max=0)
    assert torch.allclose(a, ref, atol=1e-12, rtol=0)
    assert torch.allclose(b, ref, atol=1e-12, rtol=0)


def test_general_two_orders_agree_on_rrg_workload():
    w = wl.workload(4)
    g, W = w.graphs[0], w.widths_sets[0]
    sW = torch.tensor(np.random.default_rng(2).choice([-1.0, 1.0], size=(3, len(W))))
    a = general.log_zr_general(g.n, g.ei, g.ej, g.J, 1.0, W, sW, enum_max=0)
    b = general.log_zr_general(g.n, g.ei, g.ej, g.J, 1.0, W, sW, enum_max=0, order_rule="min_degree_high")
    c = general.log_zr_general(g.n, g.ei, g.ej, g.J, 1.0, W, sW, enum_max=12)
    assert torch.allclose(a, b, atol=1e-11, rtol=0)
    assert torch.allclose(a, c, atol=1e-11, rtol=0)


def test_beta_derivative_is_minus_mean_energy():
    # d log Z_R / d beta = <-E(s, r)>_{r|s}: autograd through the strip
    # transfer matrix, enumeration, and central differences.
    g = wl.lattice(5, 4, "gauss", 8)
    W = wl.width_columns(5, 4, [2])
    sW = torch.tensor(np.random.default_rng(4).choice([-1.0, 1.0], size=(4, len(W))))
    beta = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    lzr = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, beta, W, sW, 5)
    d_auto = torch.stack([torch.autograd.grad(lzr[b], beta, retain_graph=True)[0] for b in range(4)])
    R = np.setdiff1d(np.arange(g.n), W)
    rc = ising.all_configs(len(R))
    for b in range(4):
        full = torch.zeros(rc.shape[0], g.n, dtype=torch.float64)
        full[:, torch.as_tensor(R)] = rc
        full[:, torch.as_tensor(W)] = sW[b]
        E = ising.energy(g.ei, g.ej, g.J, full)
        p = torch.softmax(-0.7 * E, 0)
        assert abs(float(-(p * E).sum()) - float(d_auto[b])) < 1e-11
        f = lambda bb: float(transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, bb, W, sW[b:b + 1], 5)[0])
        assert abs((f(0.7 + 1e-5) - f(0.7 - 1e-5)) / 2e-5 - float(d_auto[b])) < 1e-7


def test_coupling_derivative_is_beta_correlation():
    g = wl.lattice(4, 4, "pm1", 9)
    W = wl.width_columns(4, 4, [1])
    sW = torch.tensor([[1.0, -1.0, -1.0, 1.0]], dtype=torch.float64)
    J = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
    lzr = transfer.log_zr_lattice(g.n, g.ei, g.ej, J, 1.0, W, sW, 4)
    (dJ,) = torch.autograd.grad(lzr[0], J)
    R = np.setdiff1d(np.arange(g.n), W)
    rc = ising.all_configs(len(R))
    full = torch.zeros(rc.shape[0], g.n, dtype=torch.float64)
    full[:, torch.as_tensor(R)] = rc
    full[:, torch.as_tensor(W)] = sW[0]
    p = torch.softmax(-ising.energy(g.ei, g.ej, g.J, full), 0)
    corr = (p[:, None] * full[:, g.ei] * full[:, g.ej]).sum(0)
    assert torch.allclose(dJ, corr, atol=1e-12)
