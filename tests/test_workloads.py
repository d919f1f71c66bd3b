"""The seeded input generators (workloads.py) against the input recipe they
implement: lattice and complete-graph edge sets, simple random regular
graphs, coupling distributions, width sets (whole columns in autoregressive
order; the region-growing generator's separation and width bound), the five
workloads' shapes, sizes and seeds, and the MADE initialisation.  CPU only."""
import math

import numpy as np
import pytest

from paper_2504_12037_gb300 import workloads as wl


def test_lattice_edges_and_couplings():
    g = wl.lattice(5, 3, "pm1", seed=1)
    assert g.n == 15 and g.m == 4 * 3 + 5 * 2  # (Lx-1) Ly horizontal + Lx (Ly-1) vertical
    edges = {(int(a), int(b)) for a, b in zip(g.ei, g.ej)}
    assert len(edges) == g.m
    for a, b in edges:  # nearest neighbours only, each once
        ya, xa, yb, xb = a // 5, a % 5, b // 5, b % 5
        assert (ya == yb and xb == xa + 1) or (xa == xb and yb == ya + 1)
    assert set(np.unique(g.J)) <= {-1.0, 1.0}
    p = wl.lattice(4, 4, "ferro", periodic=True)
    assert p.m == 2 * 16 and np.all(p.J == 1.0)  # the torus: 2 bonds per site
    a, b = wl.lattice(16, 16, "gauss", seed=7), wl.lattice(16, 16, "gauss", seed=7)
    assert np.array_equal(a.J, b.J)  # seeded
    big = wl.lattice(64, 64, "gauss", seed=3)
    assert abs(big.J.mean()) < 0.05 and abs(big.J.std() - 1.0) < 0.05


def test_sk_couplings():
    g = wl.sk(64, 5)
    assert g.topology == wl.DENSE and g.m == 64 * 63 // 2
    assert np.all(g.ei < g.ej)
    assert abs(g.J.std() * math.sqrt(64) - 1.0) < 0.05  # J ~ N(0, 1/N)


def test_random_regular_is_simple_and_regular():
    for seed in range(3):
        g = wl.random_regular(256, 3, seed)
        deg = np.bincount(np.concatenate([g.ei, g.ej]), minlength=g.n)
        assert np.all(deg == 3)
        assert np.all(g.ei != g.ej)
        keys = g.ei.astype(np.int64) * g.n + g.ej
        assert np.unique(keys).size == g.m and np.all(g.ei < g.ej)
    with pytest.raises(ValueError):
        wl.random_regular(5, 3, 0)


def test_width_columns_order():
    W = wl.width_columns(16, 16, wl.every_kth_column(16))
    assert wl.every_kth_column(16) == [3, 7, 11, 15]
    assert W.size == 64
    # column by column (increasing x), top to bottom within a column
    assert [int(v) for v in W[:3]] == [3, 3 + 16, 3 + 32] and int(W[16]) == 7


def test_greedy_width_set_separates_components_of_bounded_width():
    g = wl.random_regular(256, 3, wl.seed_for(4))
    W = wl.greedy_width_set(g, wl.seed_for(4))
    assert len(set(W.tolist())) == W.size  # each spin once
    adj = [set() for _ in range(g.n)]
    for a, b in zip(g.ei, g.ej):
        adj[a].add(int(b))
        adj[b].add(int(a))
    wset = set(W.tolist())
    R = [v for v in range(g.n) if v not in wset]
    # components of R: at most 40 spins each, min-fill elimination width <= 8
    seen = set()
    for v in R:
        if v in seen:
            continue
        comp, stack = [], [v]
        seen.add(v)
        while stack:
            u = stack.pop()
            comp.append(u)
            for x in adj[u]:
                if x not in wset and x not in seen:
                    seen.add(x)
                    stack.append(x)
        assert len(comp) <= 40
        assert wl._minfill_width(comp, adj) <= 8


def test_five_workloads_match_the_recipe():
    w1 = wl.workload(1)
    assert (w1.graphs[0].n, w1.widths_sets[0].size, w1.hidden, w1.batch, w1.betas) == (16, 4, [16], 1024, [1.0])
    w2 = wl.workload(2)
    assert len(w2.graphs) == 5 and w2.graphs[0].n == 256 and w2.widths_sets[0].size == 64
    assert w2.hidden == [128, 128] and w2.batch == 16384
    assert np.allclose(w2.betas, [0.2, 0.4, 0.6, 0.8, 1.0])
    w3 = wl.workload(3)
    assert w3.graphs[0].n == 64 and w3.widths_sets[0].size == 48 and w3.hidden == [256, 256]
    assert w3.batch == 4096 and w3.betas == [0.5, 1.0, 2.0]
    w4 = wl.workload(4)
    assert w4.graphs[0].n == 256 and w4.widths_sets[0].size == 83 and w4.batch == 8192
    w5 = wl.workload(5)
    assert len(w5.graphs) == 64 and w5.batch == 1024 and w5.betas == [0.8] * 64
    sides = sorted({g.Lx for g in w5.graphs})
    assert set(sides) <= {8, 12, 16, 24, 32} and len(sides) == 5
    for g, W in zip(w5.graphs, w5.widths_sets):
        assert g.Lx == g.Ly and W.size == (g.Lx // 4) * g.Lx
    # seeds: workload c, instance k -> 12037 + 1000 c + k
    assert wl.seed_for(5, 3) == 12037 + 5000 + 3
    assert np.array_equal(w5.graphs[3].J, wl.lattice(w5.graphs[3].Lx, w5.graphs[3].Ly, "gauss",
                                                     wl.seed_for(5, 3)).J)


def test_ferromagnet_columns():
    w = wl.ferromagnet_columns()
    assert w.graphs[0].n == 1600 and np.all(w.graphs[0].J == 1.0)
    assert w.widths_sets[0].size == 3 * 40  # columns 12, 25, 38
    assert abs(1.0 / w.betas[2] - 2.0 / math.log(1.0 + math.sqrt(2.0))) < 1e-12
    order = w.elim_orders[0]  # every spin of R once, row by row
    assert order.size == 1600 - 120 and len(set(order.tolist())) == order.size


def test_made_params_layout_and_scale():
    D, hidden = 12, [16, 8]
    p = wl.made_params(D, hidden, 3)
    assert p.dtype == np.float32 and p.size == wl.made_param_count(D, hidden)
    assert wl.made_param_count(D, hidden) == 16 * 12 + 16 + 8 * 16 + 8 + 12 * 8 + 12
    # layer 1 weights within 1/sqrt(fan_in)
    assert np.abs(p[:16 * 12]).max() <= 1.0 / math.sqrt(12) + 1e-7
    assert np.array_equal(p, wl.made_params(D, hidden, 3))
