"""Kac-Ward determinant for the zero-field Ising model on a planar lattice
(FP64, NumPy LAPACK).  Test infrastructure only.

The paper's first experiment (Sec. 4, Fig. 2) measures the relative error of
the free energy of an open 2D ferromagnet against the exact value the
Kac-Ward method gives.  This module computes that exact value for an open
Lx x Ly square lattice (spin index y*Lx + x) with arbitrary couplings, from:

* the high-temperature expansion: with K_e = beta J_e and x_e = tanh K_e,
    Z = 2^N prod_e cosh K_e * sum over even edge subsets E' of prod_{e in E'} x_e;
* the Kac-Ward identity for a graph drawn in the plane (Kac and Ward 1952;
  proved for every planar graph by Kager, Lis and Meester 2013): that sum is
  det(I - T)^(1/2), where T acts on directed edges, T[(u->v), (v->w)] =
  x_{vw} exp(i theta / 2) for w != u, theta the turning angle from direction
  u->v to v->w (0 or +-pi/2 on the square lattice), and 0 otherwise.

So ln Z = N ln 2 + sum_e ln cosh K_e + (1/2) ln det(I - T).
"""
import math

import numpy as np


def _directions(Lx, ei, ej):
    """Unit direction (dx, dy) of every undirected edge ei -> ej."""
    ei, ej = np.asarray(ei), np.asarray(ej)
    dx = (ej % Lx) - (ei % Lx)
    dy = (ej // Lx) - (ei // Lx)
    if np.any(np.abs(dx) + np.abs(dy) != 1):
        raise ValueError("edges must join nearest neighbours of an open lattice")
    return dx, dy


def kac_ward_matrix(Lx: int, Ly: int, ei, ej, J, beta) -> np.ndarray:
    """I - T over the 2E directed edges (edge e as e: ei->ej, e + E: ej->ei)."""
    ei, ej = np.asarray(ei, np.int64), np.asarray(ej, np.int64)
    E = ei.shape[0]
    x = np.tanh(beta * np.asarray(J, np.float64))
    dx, dy = _directions(Lx, ei, ej)
    tail = np.concatenate([ei, ej])
    head = np.concatenate([ej, ei])
    ddx = np.concatenate([dx, -dx])
    ddy = np.concatenate([dy, -dy])
    weight = np.concatenate([x, x])
    out = {}  # directed edges leaving each site
    for d in range(2 * E):
        out.setdefault(int(tail[d]), []).append(d)
    M = np.eye(2 * E, dtype=np.complex128)
    for d in range(2 * E):
        for f in out.get(int(head[d]), []):
            if head[f] == tail[d]:
                continue  # no immediate return along the same edge
            theta = math.atan2(ddx[d] * ddy[f] - ddy[d] * ddx[f], ddx[d] * ddx[f] + ddy[d] * ddy[f])
            M[d, f] -= weight[f] * np.exp(0.5j * theta)
    return M


def log_z_kac_ward(Lx: int, Ly: int, ei, ej, J, beta) -> float:
    """Exact ln Z of the open Lx x Ly lattice (zero field)."""
    N = Lx * Ly
    K = beta * np.asarray(J, np.float64)
    M = kac_ward_matrix(Lx, Ly, ei, ej, J, beta)
    sign, logdet = np.linalg.slogdet(M)
    # det(I - T) is real and positive for a planar graph
    if abs(sign.imag) > 1e-8 or sign.real <= 0:
        raise ValueError(f"Kac-Ward determinant has phase {sign}")
    return N * math.log(2.0) + float(np.log(np.cosh(K)).sum()) + 0.5 * float(logdet)
