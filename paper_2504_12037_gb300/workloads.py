"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only *generates inputs*: coupling graphs, couplings J and the width
set W (the partition {s} = W u R of Sec. 2, which Algorithm 1 takes as given from
"an existing method").  It contains none of the method's arithmetic (no energy,
no contraction, no network).  Every generator is deterministic in its seed
(NumPy PCG64).

Spin-glass ensembles follow Sec. 4:
  * 2D Edwards-Anderson lattices with +/-1 couplings (Viana-Bray style
    P(J=+1) = P(J=-1) = 1/2) or Gaussian couplings;
  * the Sherrington-Kirkpatrick model (Sec. 4, last paragraph), here with
    J_ij ~ N(0, 1/N);
  * random regular graphs with +/-1 couplings (Sec. 4, Fig. 3(a)-(c)).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

LATTICE2D = 0
DENSE = 1
GENERAL = 2


@dataclasses.dataclass
class Graph:
    """An Ising coupling graph: n spins, undirected edges (ei[k], ej[k], J[k])."""

    n: int
    ei: np.ndarray  # int32 [m]
    ej: np.ndarray  # int32 [m]
    J: np.ndarray  # float64 [m]
    topology: int = GENERAL
    Lx: int = 0
    Ly: int = 0
    periodic: bool = False

    @property
    def m(self) -> int:
        return int(self.ei.shape[0])


def seed_for(config: int, instance: int = 0) -> int:
    """Seed for workload `config` (1-based) and instance k: 12037 + 1000*config + k."""
    return 12037 + 1000 * config + instance


def _couplings(rng: np.random.Generator, m: int, dist: str) -> np.ndarray:
    if dist == "pm1":
        return rng.choice(np.array([-1.0, 1.0]), size=m)
    if dist == "gauss":
        return rng.standard_normal(m)
    if dist == "ferro":
        return np.ones(m)
    raise ValueError(f"unknown coupling distribution {dist!r}")


def lattice(Lx: int, Ly: int, dist: str, seed: int = 0, periodic: bool = False) -> Graph:
    """Lx columns by Ly rows; spin index = y*Lx + x.

    Edge order: all horizontal bonds (x,y)-(x+1,y) row by row, then all vertical
    bonds (x,y)-(x,y+1) row by row.  With `periodic`, wrap-around bonds are added
    at the end of each family (only when the side is > 2).
    """
    ei: List[int] = []
    ej: List[int] = []
    for y in range(Ly):
        for x in range(Lx - 1):
            ei.append(y * Lx + x)
            ej.append(y * Lx + x + 1)
        if periodic and Lx > 2:
            ei.append(y * Lx + Lx - 1)
            ej.append(y * Lx)
    for y in range(Ly - 1):
        for x in range(Lx):
            ei.append(y * Lx + x)
            ej.append((y + 1) * Lx + x)
    if periodic and Ly > 2:
        for x in range(Lx):
            ei.append((Ly - 1) * Lx + x)
            ej.append(x)
    rng = np.random.default_rng(seed)
    J = _couplings(rng, len(ei), dist)
    return Graph(Lx * Ly, np.asarray(ei, np.int32), np.asarray(ej, np.int32), J,
                 LATTICE2D, Lx, Ly, periodic)


def sk(n: int, seed: int) -> Graph:
    """Fully connected graph, every pair i<j once, J_ij ~ N(0, 1/n)."""
    iu, ju = np.triu_indices(n, k=1)
    rng = np.random.default_rng(seed)
    J = rng.standard_normal(iu.shape[0]) / np.sqrt(n)
    return Graph(n, iu.astype(np.int32), ju.astype(np.int32), J, DENSE)


def random_regular(n: int, d: int, seed: int, dist: str = "pm1") -> Graph:
    """Random d-regular graph by configuration-model pairing; a pairing with a
    self-loop or a repeated edge is rejected and redrawn.  Couplings from `dist`."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    rng = np.random.default_rng(seed)
    for _ in range(10000):
        stubs = np.repeat(np.arange(n), d)
        rng.shuffle(stubs)
        a, b = stubs[0::2], stubs[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        keys = lo.astype(np.int64) * n + hi
        if np.unique(keys).shape[0] != keys.shape[0]:
            continue
        order = np.argsort(keys)
        lo, hi = lo[order], hi[order]
        J = _couplings(rng, lo.shape[0], dist)
        return Graph(n, lo.astype(np.int32), hi.astype(np.int32), J, GENERAL)
    raise RuntimeError("could not draw a simple random regular graph")


def width_columns(Lx: int, Ly: int, cols: Sequence[int]) -> np.ndarray:
    """Width set made of whole lattice columns, in autoregressive order:
    column by column (increasing x), top to bottom within a column."""
    return np.asarray([y * Lx + x for x in sorted(cols) for y in range(Ly)], np.int32)


def every_kth_column(L: int, k: int = 4) -> List[int]:
    """0-indexed columns c with c % k == k-1 (every k-th column)."""
    return [c for c in range(L) if c % k == k - 1]


# ---------------------------------------------------------------------------
# Greedy width set for general graphs (input choice; Algorithm 1 step 1 takes W
# as given).  Elimination width is the usual min-fill heuristic on the graph.
# ---------------------------------------------------------------------------

def _adjacency(g: Graph) -> List[set]:
    adj = [set() for _ in range(g.n)]
    for a, b in zip(g.ei.tolist(), g.ej.tolist()):
        adj[a].add(b)
        adj[b].add(a)
    return adj


def _components(nodes: Sequence[int], adj: List[set]) -> List[List[int]]:
    nodes_set = set(nodes)
    seen = set()
    comps = []
    for v in sorted(nodes_set):
        if v in seen:
            continue
        stack = [v]
        seen.add(v)
        comp = []
        while stack:
            u = stack.pop()
            comp.append(u)
            for w in adj[u]:
                if w in nodes_set and w not in seen:
                    seen.add(w)
                    stack.append(w)
        comps.append(sorted(comp))
    return comps


def _minfill_width(comp: Sequence[int], adj: List[set]) -> int:
    """Largest neighbourhood size met while eliminating by min-fill."""
    cs = set(comp)
    g = {v: set(u for u in adj[v] if u in cs) for v in comp}
    width = 0
    while g:
        best, best_fill = None, None
        for v in sorted(g):
            nb = list(g[v])
            fill = 0
            for i in range(len(nb)):
                for j in range(i + 1, len(nb)):
                    if nb[j] not in g[nb[i]]:
                        fill += 1
            if best_fill is None or fill < best_fill:
                best, best_fill = v, fill
        nb = g.pop(best)
        width = max(width, len(nb))
        for a in nb:
            g[a].discard(best)
            g[a].update(u for u in nb if u != a)
    return width


def greedy_width_set(g: Graph, seed: int, max_width: int = 8, min_size: int = 4,
                     max_size: int = 40) -> np.ndarray:
    """Greedy region growing.  Repeatedly start at the lowest-index unassigned
    spin, grow a connected region of a target size drawn uniformly from
    [min_size, max_size] (each step adds the free neighbour with the most links
    into the region, ties to the lower index), then put every free neighbour of
    the region into W.  Regions are therefore separated by W and are the
    leftover components; any region whose min-fill width exceeds max_width
    loses its highest-degree spin to W until it fits.  The returned order is the
    order in which spins entered W (the autoregressive order)."""
    adj = _adjacency(g)
    rng = np.random.default_rng(seed)
    state = np.zeros(g.n, np.int64)  # 0 free, 1 in a region, 2 in W
    W: List[int] = []
    regions: List[List[int]] = []
    while (state == 0).any():
        start = int(np.flatnonzero(state == 0)[0])
        target = int(rng.integers(min_size, max_size + 1))
        region = [start]
        state[start] = 1
        while len(region) < target:
            cand = {}
            for u in region:
                for v in adj[u]:
                    if state[v] == 0:
                        cand[v] = cand.get(v, 0) + 1
            if not cand:
                break
            v = max(cand, key=lambda v: (cand[v], -v))
            region.append(v)
            state[v] = 1
        for u in region:
            for v in sorted(adj[u]):
                if state[v] == 0:
                    state[v] = 2
                    W.append(v)
        regions.append(region)
    for region in regions:
        comps = _components(region, adj)
        while comps:
            c = comps.pop()
            if _minfill_width(c, adj) <= max_width:
                continue
            cs = set(c)
            pick = max(c, key=lambda v: (len([u for u in adj[v] if u in cs]), -v))
            W.append(pick)
            comps.extend(_components([u for u in c if u != pick], adj))
    return np.asarray(W, np.int32)


# ---------------------------------------------------------------------------
# The five workloads (graph, width set, MADE hidden widths, batch, betas).
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    graphs: List[Graph]
    widths_sets: List[np.ndarray]
    hidden: List[int]
    batch: int
    betas: List[float]
    elim_orders: Optional[List[np.ndarray]] = None  # R's elimination order per instance (GENERAL graphs)


def workload(config: int, n_instances: Optional[int] = None) -> Workload:
    """The synthetic workloads.  Instances of one workload are (graph, beta)
    pairs that run side by side in one launch."""
    if config == 1:
        g = lattice(4, 4, "pm1", seed_for(1))
        W = width_columns(4, 4, [1])
        return Workload("ea_pm1_4x4_open_col1", [g], [W], [16], 1024, [1.0])
    if config == 2:
        g = lattice(16, 16, "gauss", seed_for(2))
        W = width_columns(16, 16, every_kth_column(16))
        betas = [k / 5.0 for k in range(1, 6)]
        return Workload("ea_gauss_16x16_open_every4th_col", [g] * 5, [W] * 5, [128, 128],
                        16384, betas)
    if config == 3:
        g = sk(64, seed_for(3))
        W = np.arange(48, dtype=np.int32)
        return Workload("sk_n64_w48_r16", [g] * 3, [W] * 3, [256, 256], 4096, [0.5, 1.0, 2.0])
    if config == 4:
        g = random_regular(256, 3, seed_for(4))
        W = greedy_width_set(g, seed_for(4))
        return Workload("rrg_n256_d3_pm1_greedy_tw8", [g], [W], [128, 128], 8192, [1.0])
    if config == 5:
        n = 64 if n_instances is None else n_instances
        rng = np.random.default_rng(seed_for(5))
        sizes = rng.choice(np.array([8, 12, 16, 24, 32]), size=n)
        graphs, Ws = [], []
        for k in range(n):
            L = int(sizes[k])
            graphs.append(lattice(L, L, "gauss", seed_for(5, k)))
            Ws.append(width_columns(L, L, every_kth_column(L)))
        return Workload("ea_gauss_multi_instance_train", graphs, Ws, [128, 128], 1024,
                        [0.8] * n)
    raise ValueError(f"unknown workload {config}")


def ferromagnet_columns(L: int = 40, period: int = 13, hidden: Sequence[int] = (256, 256),
                        batch: int = 1000) -> Workload:
    """The paper's first experiment (Sec. 4, Fig. 2): the open L x L
    ferromagnet (J = 1) at T = 1, 2, T_c, 3, 4, 5 (T_c = 2 / ln(1 + sqrt 2),
    Onsager's critical temperature), one instance per temperature; W = every
    `period`-th column (columns c with c % period == period - 1), which leaves
    strips of period - 1 columns.  With period > 5 the strips are wider than
    the per-thread strip contraction takes: the plan is an elimination plan
    (each strip eliminated row by row, elimination width = strip width, the
    order given here) and the forward contraction runs the wide-strip kernel."""
    g = lattice(L, L, "ferro", 0)
    cols = every_kth_column(L, period)
    W = width_columns(L, L, cols)
    order = None
    if period > 5:
        wset = set(int(v) for v in W)
        order = np.asarray([y * L + x for y in range(L) for x in range(L) if y * L + x not in wset], np.int32)
    temps = [1.0, 2.0, 2.0 / np.log(1.0 + np.sqrt(2.0)), 3.0, 4.0, 5.0]
    n = len(temps)
    return Workload(f"ferro_{L}x{L}_open_every{period}th_col", [g] * n, [W] * n, list(hidden), batch,
                    [float(1.0 / T) for T in temps], None if order is None else [order] * n)


# ---------------------------------------------------------------------------
# Network parameters (seeded initial values; layout of the C-ABI: per layer
# W [out][in] row-major, then b [out]).
# ---------------------------------------------------------------------------

def made_param_count(D: int, hidden: Sequence[int]) -> int:
    sz = [D] + list(hidden) + [D]
    return sum(sz[l + 1] * sz[l] + sz[l + 1] for l in range(len(sz) - 1))


def made_params(D: int, hidden: Sequence[int], seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (PyTorch's
    default Linear initialisation), times `scale`, as float32."""
    rng = np.random.default_rng(seed)
    sz = [D] + list(hidden) + [D]
    parts = []
    for l in range(len(sz) - 1):
        bound = scale / np.sqrt(sz[l])
        parts.append(rng.uniform(-bound, bound, size=sz[l + 1] * sz[l]))
        parts.append(rng.uniform(-bound, bound, size=sz[l + 1]))
    return np.concatenate(parts).astype(np.float32)
