"""Pins for oracle.transfer: brute force, Kaufman's closed form, Onsager."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import ising, transfer
from paper_2504_12037_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("Lx,Ly,dist,beta", [(4, 4, "gauss", 0.7), (3, 5, "pm1", 1.0), (5, 3, "gauss", 1.3)])
def test_rowtm_and_helical_equal_brute_force(Lx, Ly, dist, beta):
    g = wl.lattice(Lx, Ly, dist, 11)
    ref = float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, beta))
    assert abs(float(transfer.log_z_rowtm(Lx, Ly, g.ei, g.ej, g.J, beta)) - ref) < 1e-12 * abs(ref)
    assert abs(float(transfer.log_z_helical(Lx, Ly, g.ei, g.ej, g.J, beta)) - ref) < 1e-12 * abs(ref)


def test_helical_equals_rowtm_8x8():
    g = wl.lattice(8, 8, "gauss", 12)
    a = float(transfer.log_z_rowtm(8, 8, g.ei, g.ej, g.J, 0.9))
    b = float(transfer.log_z_helical(8, 8, g.ei, g.ej, g.J, 0.9))
    assert abs(a - b) < 1e-11 * abs(a)


@pytest.mark.parametrize("Lx,Ly", [(4, 4), (4, 3), (3, 4), (5, 3)])
@pytest.mark.parametrize("beta", [0.25, 0.6, 1.1])
def test_kaufman_equals_brute_force_on_small_tori(Lx, Ly, beta):
    g = wl.lattice(Lx, Ly, "ferro", periodic=True)
    ref = float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, beta))
    assert abs(transfer.kaufman_log_z(Ly, Lx, beta) - ref) < 1e-11 * abs(ref)


@pytest.mark.parametrize("Lx,Ly", [(6, 6), (7, 5)])
@pytest.mark.parametrize("beta", [0.3, 0.7])
def test_torus_rowtm_equals_kaufman(Lx, Ly, beta):
    g = wl.lattice(Lx, Ly, "ferro", periodic=True)
    a = float(transfer.log_z_rowtm(Lx, Ly, g.ei, g.ej, g.J, beta))
    assert abs(a - transfer.kaufman_log_z(Ly, Lx, beta)) < 1e-11 * abs(a)


def test_kaufman_large_torus_approaches_onsager():
    # Above T_c the finite-size correction is exponentially small; below T_c
    # the torus keeps the two ordered states, f_L = f_inf - T ln 2 / N + o(e^-L).
    L = 96
    N = L * L
    for T, shift in ((3.0, 0.0), (1.5, -1.5 * math.log(2) / N)):
        beta = 1.0 / T
        f_k = -transfer.kaufman_log_z(L, L, beta) / (beta * N)
        assert abs(f_k - (transfer.onsager_f(beta) + shift)) < 1e-9


def test_kaufman_gamma0_changes_sign_at_paper_tc():
    with open(os.path.join(GOLDEN, "critical_temperature.txt")) as fh:
        tc = float([l for l in fh if not l.startswith("#")][0])
    g0 = lambda T: 2 / T + math.log(math.tanh(1 / T))
    assert g0(tc - 1e-4) > 0 > g0(tc + 1e-4)  # positive in the ordered phase
    # and the exact value 2/ln(1+sqrt 2) agrees with the paper's 5 decimals
    assert abs(2 / math.log(1 + math.sqrt(2)) - tc) < 1e-5


def test_strip_tm_equals_enumeration_cfg1():
    w = wl.workload(1)
    g, W = w.graphs[0], w.widths_sets[0]
    sW = ising.all_configs(len(W))
    a = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, 1.0, W, sW, g.Lx)
    b = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 1.0, W, sW)
    assert torch.allclose(a, b, atol=1e-12, rtol=0)


@pytest.mark.parametrize("Lx,Ly,cols", [(5, 4, [2]), (7, 3, [3]), (6, 3, [0, 4]), (4, 5, [3])])
def test_strip_tm_equals_enumeration_other_shapes(Lx, Ly, cols):
    g = wl.lattice(Lx, Ly, "gauss", 21)
    W = wl.width_columns(Lx, Ly, cols)
    rng = np.random.default_rng(3)
    sW = torch.tensor(rng.choice([-1.0, 1.0], size=(6, len(W))))
    a = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, 0.8, W, sW, Lx)
    b = ising.log_zr_enum(g.n, g.ei, g.ej, g.J, 0.8, W, sW)
    assert torch.allclose(a, b, atol=1e-11, rtol=0)


def test_strip_factorisation_16x16_matches_helical_at_high_temperature():
    # Sum over W of exp(log Z_R) = Z, checked at tiny beta where a modest
    # importance sample over uniform W states is essentially exact.
    g = wl.lattice(8, 4, "gauss", 5)
    W = wl.width_columns(8, 4, [3])
    sW = ising.all_configs(4)
    lzr = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, 0.5, W, sW, 8)
    ref = float(transfer.log_z_helical(8, 4, g.ei, g.ej, g.J, 0.5))
    assert abs(float(torch.logsumexp(lzr, 0)) - ref) < 1e-12 * abs(ref)
