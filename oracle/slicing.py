"""Width of a sliced network (Sec. 2: width set W, contraction width w_u).
Test infrastructure only.

Removing the spins of W from the graph leaves the network on R.  Eliminating
a spin v of R (summing it out) leaves one factor over the spins adjacent to v
at that moment -- its neighbours in the graph where every earlier elimination
joined its own neighbours pairwise.  The width of an elimination order is the
largest number of spins in such a factor; the smallest width over all orders
is the treewidth of the graph on R, and w_u = 1 means R is a forest (W a
feedback vertex set).

  elimination_width   the width of one given order, by direct simulation.
  treewidth           the smallest width over all orders, by dynamic
                      programming over subsets of eliminated spins (small
                      graphs only): TW(S) = min over v in S of
                      max(TW(S - v), |Q(S - v, v)|), where Q(S, v) are the
                      spins outside S + v reachable from v through S.
  min_width_set       the smallest W with treewidth(G - W) <= w_u, by
                      enumerating subsets in order of size (tiny graphs).
"""
from itertools import combinations
from typing import Iterable, List, Optional, Sequence, Set


def _adjacency(n: int, ei: Sequence[int], ej: Sequence[int], removed: Iterable[int] = ()) -> List[Set[int]]:
    gone = set(int(x) for x in removed)
    adj = [set() for _ in range(n)]
    for a, b in zip(ei, ej):
        a, b = int(a), int(b)
        if a in gone or b in gone:
            continue
        adj[a].add(b)
        adj[b].add(a)
    return adj


def elimination_width(n: int, ei, ej, removed: Iterable[int], order: Sequence[int]) -> int:
    """Largest factor (neighbour count at elimination) when the spins of
    `order` are summed out in turn from the graph without `removed`."""
    adj = _adjacency(n, ei, ej, removed)
    width = 0
    for v in order:
        v = int(v)
        nb = set(adj[v])
        width = max(width, len(nb))
        for a in nb:
            adj[a] |= nb
            adj[a].discard(a)
            adj[a].discard(v)
        adj[v] = set()
    return width


def _q_size(adj: List[Set[int]], S: int, v: int) -> int:
    """|Q(S, v)|: spins outside S and v reachable from v through S (S a bit mask)."""
    seen = {v}
    stack = [v]
    out = set()
    while stack:
        u = stack.pop()
        for w in adj[u]:
            if w in seen:
                continue
            seen.add(w)
            if (S >> w) & 1:
                stack.append(w)
            else:
                out.add(w)
    return len(out)


def treewidth(n: int, ei, ej, removed: Iterable[int] = ()) -> int:
    """Treewidth of the graph on the spins not removed (0 for no edges)."""
    gone = set(int(x) for x in removed)
    keep = [v for v in range(n) if v not in gone]
    if not keep:
        return 0
    loc = {v: k for k, v in enumerate(keep)}
    m = len(keep)
    if m > 18:
        raise ValueError("treewidth by subset DP is for at most 18 spins")
    adj = [set() for _ in range(m)]
    for a, b in zip(ei, ej):
        a, b = int(a), int(b)
        if a in loc and b in loc:
            adj[loc[a]].add(loc[b])
            adj[loc[b]].add(loc[a])
    INF = 10 ** 9
    tw = [INF] * (1 << m)
    tw[0] = -1  # no spin eliminated yet
    for S in range(1, 1 << m):
        best = INF
        x = S
        while x:
            low = x & -x
            v = low.bit_length() - 1
            x ^= low
            rest = S ^ low
            cand = max(tw[rest], _q_size(adj, rest, v))
            if cand < best:
                best = cand
        tw[S] = best
    return max(tw[(1 << m) - 1], 0)


def min_width_set(n: int, ei, ej, w_u: int, max_size: Optional[int] = None) -> List[int]:
    """A smallest W (lowest indices first among equals) with
    treewidth(G - W) <= w_u."""
    top = n if max_size is None else max_size
    for k in range(0, top + 1):
        for W in combinations(range(n), k):
            if treewidth(n, ei, ej, W) <= w_u:
                return list(W)
    raise ValueError("no width set within max_size")
