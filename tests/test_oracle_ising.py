"""Pins for oracle.ising: closed forms and invariants (no GPU)."""
import math

import numpy as np
import torch

from oracle import ising
from paper_2504_12037_gb300 import workloads as wl


def test_open_chain_closed_form():
    # A 1D open chain (a tree) has Z = 2 prod_e 2 cosh(beta J_e).
    rng = np.random.default_rng(0)
    n = 12
    J = rng.standard_normal(n - 1)
    ei, ej = np.arange(n - 1), np.arange(1, n)
    beta = 0.8
    expect = math.log(2) + sum(math.log(2 * math.cosh(beta * j)) for j in J)
    assert abs(float(ising.log_z_brute(n, ei, ej, J, beta)) - expect) < 1e-12


def test_random_tree_closed_form():
    rng = np.random.default_rng(1)
    n = 13
    parent = [int(rng.integers(0, k)) for k in range(1, n)]
    ei, ej = np.array(parent), np.arange(1, n)
    J = rng.standard_normal(n - 1) * 2
    beta = 0.6
    expect = math.log(2) + sum(math.log(2 * math.cosh(beta * j)) for j in J)
    assert abs(float(ising.log_z_brute(n, ei, ej, J, beta)) - expect) < 1e-12


def test_energy_all_up_and_sign():
    g = wl.lattice(4, 4, "gauss", 3)
    up = torch.ones(1, g.n, dtype=torch.float64)
    assert abs(float(ising.energy(g.ei, g.ej, g.J, up)[0]) + g.J.sum()) < 1e-12
    s = torch.tensor(np.random.default_rng(2).choice([-1.0, 1.0], size=(5, g.n)))
    E = ising.energy(g.ei, g.ej, g.J, s)
    direct = torch.tensor([-sum(g.J[k] * s[b, g.ei[k]] * s[b, g.ej[k]] for k in range(g.m)) for b in range(5)])
    assert torch.allclose(E, direct, atol=1e-12)


def test_width_set_factorisation_4x4():
    # Eq. 3: sum over all 2^|W| width-set states of exp(log Z_R(s)) is Z.
    w = wl.workload(1)
    g, W = w.graphs[0], w.widths_sets[0]
    beta = 1.0
    sW = ising.all_configs(len(W))
    lzr = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, beta, W, sW)
    lz = ising.log_z_brute(g.n, g.ei, g.ej, g.J, beta)
    assert abs(float(torch.logsumexp(lzr, 0)) - float(lz)) < 1e-12 * abs(float(lz))


def test_zero_field_flip_symmetry():
    g = wl.lattice(4, 4, "pm1", 7)
    W = wl.width_columns(4, 4, [1])
    sW = ising.all_configs(4)
    a = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 0.9, W, sW)
    b = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 0.9, W, -sW)
    assert torch.allclose(a, b, atol=1e-12)


def test_components_of_column_width_set():
    g = wl.lattice(16, 16, "gauss", 1)
    W = wl.width_columns(16, 16, wl.every_kth_column(16))
    comps = ising.components(g.n, g.ei, g.ej, W)
    assert len(comps) == 4 and all(len(c) == 48 for c in comps)
