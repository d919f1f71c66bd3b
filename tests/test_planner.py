"""The width-set finder tnvan_find_width_set (Sec. 2: order search, dynamic
slicing, random return of sliced spins), called through the C-ABI on the
host (no GPU), checked with oracle/slicing.py: the returned order of R has
exactly the reported width (<= w_u), W and R partition the spins, w_u = 1
leaves a forest, closed forms (complete graphs, cycles, trees), and the
smallest width sets of tiny graphs by brute force."""
import os

import networkx as nx
import numpy as np
import pytest

from oracle import slicing as sl
from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(tv.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()


def _g(G):
    G = nx.convert_node_labels_to_integers(G)
    e = list(G.edges())
    return G.number_of_nodes(), np.array([a for a, _ in e], np.int32), np.array([b for _, b in e], np.int32)


def _check(n, ei, ej, wu, W, order, width):
    W = [int(x) for x in W]
    assert len(set(W)) == len(W) and all(0 <= x < n for x in W)
    assert sorted(W + [int(x) for x in order]) == list(range(n))
    assert sl.elimination_width(n, ei, ej, W, order) == width
    assert width <= wu
    if wu == 1:
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(ei.tolist(), ej.tolist()))
        G.remove_nodes_from(W)
        assert nx.is_forest(G)


@pytest.mark.parametrize("mode", [tv.SLICE_FIXED, tv.SLICE_GREEDY, tv.SLICE_BEST])
@pytest.mark.parametrize("graph,wu", [
    ("rrg300d4", 1), ("rrg300d4", 3), ("rrg300d4", 8), ("rrg256d3", 8), ("lattice16", 3), ("sk24", 5),
])
def test_finder_output_is_valid(graph, wu, mode):
    if graph == "rrg300d4":
        g = wl.random_regular(300, 4, 12037)
    elif graph == "rrg256d3":
        g = wl.random_regular(256, 3, 12037)
    elif graph == "lattice16":
        g = wl.lattice(16, 16, "gauss", seed=12037)
    else:
        g = wl.sk(24, 12037)
    ei, ej = np.asarray(g.ei, np.int32), np.asarray(g.ej, np.int32)
    W, order, width, tag = tv.find_width_set(g.n, ei, ej, wu, restarts=2, seed=5, mode=mode)
    _check(g.n, ei, ej, wu, W, order, width)
    if mode == tv.SLICE_FIXED:
        assert tag % 2 == 0
    if mode == tv.SLICE_GREEDY:
        assert tag % 2 == 1


def test_finder_is_deterministic_and_best_mode_is_no_worse():
    g = wl.random_regular(300, 4, 12037)
    a = tv.find_width_set(g.n, g.ei, g.ej, 3, restarts=3, seed=9)
    b = tv.find_width_set(g.n, g.ei, g.ej, 3, restarts=3, seed=9)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2:] == b[2:]
    f = tv.find_width_set(g.n, g.ei, g.ej, 3, restarts=3, seed=9, mode=tv.SLICE_FIXED)
    gr = tv.find_width_set(g.n, g.ei, g.ej, 3, restarts=3, seed=9, mode=tv.SLICE_GREEDY)
    assert len(a[0]) == min(len(f[0]), len(gr[0]))


@pytest.mark.parametrize("n,wu", [(8, 1), (8, 3), (10, 6), (12, 11)])
def test_complete_graph_closed_form(n, wu):
    m, ei, ej = _g(nx.complete_graph(n))
    W, order, width, _ = tv.find_width_set(m, ei, ej, wu)
    assert len(W) == max(n - 1 - wu, 0)
    _check(m, ei, ej, wu, W, order, width)


def test_cycles_and_trees():
    m, ei, ej = _g(nx.cycle_graph(20))
    W, order, width, _ = tv.find_width_set(m, ei, ej, 1)
    assert len(W) == 1 and width == 1
    W, order, width, _ = tv.find_width_set(m, ei, ej, 2)
    assert len(W) == 0 and width == 2
    m, ei, ej = _g(nx.balanced_tree(3, 4))
    W, order, width, _ = tv.find_width_set(m, ei, ej, 1)
    assert len(W) == 0 and width == 1
    _check(m, ei, ej, 1, W, order, width)
    # isolated spins and no edges at all
    W, order, width, _ = tv.find_width_set(5, np.zeros(0, np.int32), np.zeros(0, np.int32), 0)
    assert len(W) == 0 and width == 0 and sorted(order.tolist()) == list(range(5))


def test_against_brute_force_on_tiny_graphs():
    """Heuristic: never below the optimum (that would be an invalid W), and
    within one spin of it on these graphs."""
    gaps = []
    for seed in range(12):
        G = nx.gnm_random_graph(10, 17, seed=seed)
        n, ei, ej = _g(G)
        for wu in (1, 2):
            best = len(sl.min_width_set(n, ei, ej, wu))
            W, order, width, _ = tv.find_width_set(n, ei, ej, wu, restarts=4, seed=seed)
            _check(n, ei, ej, wu, W, order, width)
            assert len(W) >= best
            gaps.append(len(W) - best)
    assert max(gaps) <= 1


def test_bad_arguments_are_rejected():
    L = tv.lib()
    ei = np.array([0, 1], np.int32)
    ej = np.array([1, 1], np.int32)  # self-loop
    with pytest.raises(tv.TnvanError):
        tv.find_width_set(2, ei, ej, 1)
    with pytest.raises(tv.TnvanError):
        tv.find_width_set(3, np.array([0], np.int32), np.array([5], np.int32), 1)
    with pytest.raises(tv.TnvanError):
        tv.find_width_set(3, np.array([0], np.int32), np.array([1], np.int32), 1, restarts=0)
    with pytest.raises(tv.TnvanError):
        tv.find_width_set(3, np.array([0], np.int32), np.array([1], np.int32), 1, mode=4)
    with pytest.raises(tv.TnvanError):
        tv.find_width_set(3, np.array([0], np.int32), np.array([1], np.int32), 1, anneal=-1)
    assert L.tnvan_find_width_set(0, 0, None, None, 1, 1, 0, 3, 0, None, None, None) == tv.E_ARG


@pytest.mark.parametrize("graph,wu", [("rrg300d4", 3), ("rrg300d4", 8), ("rrg256d3", 6)])
def test_annealing_keeps_valid_sets_and_never_grows_them(graph, wu):
    g = wl.random_regular(300, 4, 12037) if graph == "rrg300d4" else wl.random_regular(256, 3, 12037)
    ei, ej = np.asarray(g.ei, np.int32), np.asarray(g.ej, np.int32)
    base = tv.find_width_set(g.n, ei, ej, wu, restarts=2, seed=7)
    W, order, width, _ = tv.find_width_set(g.n, ei, ej, wu, restarts=2, seed=7, anneal=400)
    _check(g.n, ei, ej, wu, W, order, width)
    assert len(W) <= len(base[0])
    again = tv.find_width_set(g.n, ei, ej, wu, restarts=2, seed=7, anneal=400)
    assert np.array_equal(again[0], W) and np.array_equal(again[1], order)


def test_zero_width_leaves_an_independent_set():
    """w_u = 0: every spin of R is summed alone, so R has no bonds and W is a
    vertex cover; on bipartite graphs the smallest cover has the size of a
    maximum matching (Konig), which the brute force confirms."""
    for seed in range(6):
        G = nx.bipartite.random_graph(5, 5, 0.4, seed=seed)
        n, ei, ej = _g(G)
        W, order, width, _ = tv.find_width_set(n, ei, ej, 0, restarts=4, seed=seed)
        _check(n, ei, ej, 0, W, order, width)
        Wset = set(int(x) for x in W)
        assert all(a in Wset or b in Wset for a, b in zip(ei.tolist(), ej.tolist()))
        best = len(sl.min_width_set(n, ei, ej, 0))
        matching = len(nx.max_weight_matching(nx.convert_node_labels_to_integers(G), maxcardinality=True))
        assert best == matching
        assert best <= len(W) <= best + 1
