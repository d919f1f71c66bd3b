"""Pins for oracle.kacward (the exact free energy of the paper's 2D lattice
experiment, Sec. 4): brute-force enumeration, the single-site transfer matrix,
the open-chain closed form and the gauge symmetry J -> -J of a bipartite
lattice."""
import math

import numpy as np
import pytest

from oracle import ising, kacward, transfer
from paper_2504_12037_gb300 import workloads as wl


@pytest.mark.parametrize("Lx,Ly,dist,seed", [(4, 4, "gauss", 1), (3, 5, "gauss", 2), (4, 4, "pm1", 3),
                                             (5, 3, "gauss", 4), (2, 2, "gauss", 5)])
def test_kac_ward_equals_brute_force(Lx, Ly, dist, seed):
    g = wl.lattice(Lx, Ly, dist, seed)
    for beta in (0.3, 1.0, 2.5):
        a = kacward.log_z_kac_ward(Lx, Ly, g.ei, g.ej, g.J, beta)
        b = float(ising.log_z_brute(g.n, g.ei, g.ej, g.J, beta))
        assert abs(a - b) <= 1e-12 * abs(b)


def test_kac_ward_equals_helical_transfer_matrix():
    for Lx, Ly, seed in ((12, 12, 7), (10, 7, 8)):
        g = wl.lattice(Lx, Ly, "gauss", seed)
        for beta in (0.44, 1.3):
            a = kacward.log_z_kac_ward(Lx, Ly, g.ei, g.ej, g.J, beta)
            b = float(transfer.log_z_helical(Lx, Ly, g.ei, g.ej, g.J, beta))
            assert abs(a - b) <= 1e-12 * abs(b)


def test_open_chain_closed_form():
    # a 1 x L chain: Z = 2 prod_e 2 cosh(beta J_e)
    g = wl.lattice(1, 9, "gauss", 11)
    for beta in (0.2, 1.7):
        want = math.log(2.0) + sum(math.log(2 * math.cosh(beta * J)) for J in g.J)
        assert abs(kacward.log_z_kac_ward(1, 9, g.ei, g.ej, g.J, beta) - want) <= 1e-13 * abs(want)


def test_gauge_symmetry_of_the_bipartite_lattice():
    # flipping the spins of one sublattice maps J to -J on every bond: Z unchanged
    g = wl.lattice(9, 8, "gauss", 12)
    a = kacward.log_z_kac_ward(9, 8, g.ei, g.ej, g.J, 0.9)
    b = kacward.log_z_kac_ward(9, 8, g.ei, g.ej, -np.asarray(g.J), 0.9)
    assert abs(a - b) <= 1e-12 * abs(a)
