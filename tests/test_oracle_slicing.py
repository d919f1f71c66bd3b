"""Pins of oracle/slicing.py (widths of sliced networks, Sec. 2) against
textbook values: treewidths of complete, cycle, tree, grid, complete
bipartite and Petersen graphs, decycling numbers (smallest feedback vertex
sets, the w_u = 1 case), and widths of hand-checked elimination orders."""
import networkx as nx
import pytest

from oracle import slicing as sl


def _edges(G):
    e = list(G.edges())
    return [a for a, _ in e], [b for _, b in e]


def _g(G):
    G = nx.convert_node_labels_to_integers(G)
    ei, ej = _edges(G)
    return G.number_of_nodes(), ei, ej


@pytest.mark.parametrize("G,tw", [
    (nx.complete_graph(6), 5),
    (nx.cycle_graph(9), 2),
    (nx.path_graph(7), 1),
    (nx.balanced_tree(2, 2), 1),
    (nx.grid_2d_graph(3, 3), 3),
    (nx.grid_2d_graph(3, 4), 3),
    (nx.complete_bipartite_graph(3, 4), 3),
    (nx.petersen_graph(), 4),
    (nx.empty_graph(5), 0),
])
def test_treewidth_textbook_values(G, tw):
    n, ei, ej = _g(G)
    assert sl.treewidth(n, ei, ej) == tw


@pytest.mark.parametrize("G,k", [
    (nx.complete_graph(5), 3),            # K_n: n - 2
    (nx.cycle_graph(8), 1),
    (nx.balanced_tree(2, 2), 0),
    (nx.petersen_graph(), 3),             # decycling number of the Petersen graph
    (nx.complete_bipartite_graph(3, 3), 2),  # K_{m,n}, m <= n: m - 1
    (nx.grid_2d_graph(3, 3), 2),
])
def test_min_feedback_vertex_set_sizes(G, k):
    n, ei, ej = _g(G)
    W = sl.min_width_set(n, ei, ej, 1)
    assert len(W) == k
    H = nx.convert_node_labels_to_integers(G).copy()
    H.remove_nodes_from(W)
    assert nx.is_forest(H) or H.number_of_nodes() == 0


@pytest.mark.parametrize("n,wu", [(6, 1), (6, 2), (6, 4), (7, 3)])
def test_complete_graph_width_set(n, wu):
    m, ei, ej = _g(nx.complete_graph(n))
    assert len(sl.min_width_set(m, ei, ej, wu)) == n - 1 - wu


def test_elimination_width_of_given_orders():
    n, ei, ej = _g(nx.star_graph(6))          # centre 0, leaves 1..6
    assert sl.elimination_width(n, ei, ej, [], [0, 1, 2, 3, 4, 5, 6]) == 6
    assert sl.elimination_width(n, ei, ej, [], [1, 2, 3, 4, 5, 6, 0]) == 1
    assert sl.elimination_width(n, ei, ej, [0], [1, 2, 3, 4, 5, 6]) == 0
    n, ei, ej = _g(nx.cycle_graph(7))
    assert sl.elimination_width(n, ei, ej, [], [3, 0, 6, 1, 5, 2, 4]) == 2
    # removing 2 leaves the path 3-4-5-6-0-1: from an end width 1, from inside 2
    assert sl.elimination_width(n, ei, ej, [2], [3, 4, 5, 6, 0, 1]) == 1
    assert sl.elimination_width(n, ei, ej, [2], [0, 1, 3, 4, 5, 6]) == 2
    n, ei, ej = _g(nx.grid_2d_graph(3, 3))    # row-major labels
    # row by row: the frontier holds one row (3 spins) plus the next spin
    assert sl.elimination_width(n, ei, ej, [], list(range(9))) == 3
    # the centre first: its four neighbours form the factor (then a clique)
    assert sl.elimination_width(n, ei, ej, [], [4, 0, 1, 2, 3, 5, 6, 7, 8]) == 4


def test_treewidth_is_the_best_order():
    # brute force over every order of a small random graph
    from itertools import permutations
    G = nx.gnm_random_graph(7, 12, seed=3)
    n, ei, ej = _g(G)
    best = min(sl.elimination_width(n, ei, ej, [], p) for p in permutations(range(n)))
    assert sl.treewidth(n, ei, ej) == best
