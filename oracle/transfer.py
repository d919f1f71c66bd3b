"""Transfer-matrix contractions of Eq. 2 in plain dense form (FP64, torch on
the CPU, differentiable in J and beta).  Test infrastructure only.

* `log_zr_lattice`: per-sample log Z_R(s) (Eq. 4) for lattice graphs whose
  leftover components are bands of whole rows: for every component a dense
  2^w row transfer matrix is built straight from the edge list and the chain is
  multiplied row by row, renormalised by its maximum after every row.
* `log_z_rowtm`: whole-lattice ln Z by the same dense row transfer matrix
  (open, or periodic: trace of the product).
* `log_z_helical`: whole-lattice ln Z for an open lattice by the single-site
  ("helical") transfer matrix over the 2^Lx frontier states.
* `kaufman_log_z`: Kaufman's closed form (Phys. Rev. 76, 1232 (1949)) for the
  ferromagnetic m x n torus; `onsager_f`: Onsager's infinite-lattice free energy.
"""
import math

import numpy as np
import torch

from .ising import DT, all_configs, components, w_energy_term


def _edge_index(ei, ej):
    return list(zip(np.asarray(ei).tolist(), np.asarray(ej).tolist()))


def _chain(diags, verts):
    """ln of 1^T D_0 V_0 D_1 V_1 ... D_{L-1} 1 with per-row max renormalisation.
    diags[y]: [B, K] log-weights; verts[y]: [K, K] log-weights."""
    v = diags[0]
    m = v.max(dim=1, keepdim=True).values
    v = torch.exp(v - m)
    acc = m[:, 0]
    for y in range(1, len(diags)):
        v = v @ torch.exp(verts[y - 1])
        v = v * torch.exp(diags[y] - diags[y].max(dim=1, keepdim=True).values)
        acc = acc + diags[y].max(dim=1).values
        m = v.max(dim=1, keepdim=True).values
        v = v / m
        acc = acc + torch.log(m[:, 0])
    return acc + torch.log(v.sum(dim=1))


def log_zr_lattice(n, ei, ej, J, beta, W, sW: torch.Tensor, Lx: int, field=None) -> torch.Tensor:
    """log Z_R(s) = -beta E_1(s) + sum_c ln Z_c(s) (Eq. 4) for sW [B, |W|] on a
    lattice with spin index y*Lx + x.  Each leftover component must occupy the
    same columns in a run of consecutive rows.  `field` ([B] or a scalar): a
    uniform field on R, beta * field * (sum of the row's spins) in every row."""
    J = torch.as_tensor(J, dtype=DT) if not torch.is_tensor(J) else J
    sW = sW.to(DT)
    B = sW.shape[0]
    Wl = [int(w) for w in np.asarray(W).tolist()]
    wpos = {w: k for k, w in enumerate(Wl)}
    edges = _edge_index(ei, ej)
    total = w_energy_term(ei, ej, J, beta, W, sW)
    for comp in components(n, ei, ej, W):
        rows = sorted(set(v // Lx for v in comp))
        cols = sorted(set(v % Lx for v in comp if v // Lx == rows[0]))
        if rows != list(range(rows[0], rows[-1] + 1)):
            raise ValueError("component rows are not consecutive")
        for v in comp:
            if v % Lx not in cols:
                raise ValueError("component is not a band of whole rows")
        w = len(cols)
        cpos = {c: k for k, c in enumerate(cols)}
        X = all_configs(w)  # [2^w, w]
        diags = [torch.zeros(B, 2 ** w, dtype=DT) for _ in rows]
        if field is not None:
            fb = field[:, None] if torch.is_tensor(field) and field.dim() > 0 else field
            diags = [d + beta * fb * X.sum(1)[None, :] for d in diags]
        verts = [torch.zeros(2 ** w, 2 ** w, dtype=DT) for _ in rows[:-1]]
        cset = set(comp)
        for e, (a, b) in enumerate(edges):
            ina, inb = a in cset, b in cset
            if not (ina or inb):
                continue
            if ina and inb:
                ya, yb = a // Lx, b // Lx
                if ya == yb:
                    k = ya - rows[0]
                    diags[k] = diags[k] + beta * J[e] * (X[:, cpos[a % Lx]] * X[:, cpos[b % Lx]])[None, :]
                elif abs(ya - yb) == 1:
                    lo, hi = (a, b) if ya < yb else (b, a)
                    k = lo // Lx - rows[0]
                    verts[k] = verts[k] + beta * J[e] * torch.outer(X[:, cpos[lo % Lx]], X[:, cpos[hi % Lx]])
                else:
                    raise ValueError("bond skips rows")
            else:
                r, wv = (a, b) if ina else (b, a)
                if wv not in wpos:
                    raise ValueError("component touches a spin outside W")
                k = r // Lx - rows[0]
                diags[k] = diags[k] + beta * J[e] * sW[:, wpos[wv]][:, None] * X[:, cpos[r % Lx]][None, :]
        total = total + _chain(diags, verts)
    return total


def log_z_rowtm(Lx: int, Ly: int, ei, ej, J, beta) -> torch.Tensor:
    """Whole-lattice ln Z by dense 2^Lx row transfer matrices.  Bonds between
    row Ly-1 and row 0 (periodic) make it a trace."""
    J = torch.as_tensor(J, dtype=DT) if not torch.is_tensor(J) else J
    X = all_configs(Lx)
    K = 2 ** Lx
    diag = [torch.zeros(K, dtype=DT) for _ in range(Ly)]
    vert = [torch.zeros(K, K, dtype=DT) for _ in range(Ly)]
    wrap = False
    for e, (a, b) in enumerate(_edge_index(ei, ej)):
        ya, yb, xa, xb = a // Lx, b // Lx, a % Lx, b % Lx
        if ya == yb:
            diag[ya] = diag[ya] + beta * J[e] * X[:, xa] * X[:, xb]
        elif yb == ya + 1 or ya == yb + 1:
            lo, hi = (a, b) if ya < yb else (b, a)
            vert[lo // Lx] = vert[lo // Lx] + beta * J[e] * torch.outer(X[:, lo % Lx], X[:, hi % Lx])
        else:  # wrap bond between row Ly-1 and row 0
            top, bot = (a, b) if ya == Ly - 1 else (b, a)
            vert[Ly - 1] = vert[Ly - 1] + beta * J[e] * torch.outer(X[:, top % Lx], X[:, bot % Lx])
            wrap = True
    if not wrap:
        return _chain([d[None, :] for d in diag], vert[:-1])[0]
    M = torch.eye(K, dtype=DT)
    acc = torch.zeros((), dtype=DT)
    for y in range(Ly):
        M = (M * torch.exp(diag[y])[None, :]) @ torch.exp(vert[y])
        m = M.abs().max()
        M = M / m
        acc = acc + torch.log(m)
    return acc + torch.log(torch.trace(M))


def log_z_helical(Lx: int, Ly: int, ei, ej, J, beta) -> torch.Tensor:
    """ln Z of an open Lx x Ly lattice by the single-site transfer matrix: the
    state is the frontier of Lx spins (bit x = spin in column x, bit set = -1),
    and sites are added in row-major order."""
    J = torch.as_tensor(J, dtype=DT) if not torch.is_tensor(J) else J
    bond = {}
    for e, (a, b) in enumerate(_edge_index(ei, ej)):
        bond[(min(a, b), max(a, b))] = e
    X = all_configs(Lx)
    lw = torch.zeros(2 ** Lx, dtype=DT)
    for x in range(Lx - 1):
        e = bond.get((x, x + 1))
        if e is not None:
            lw = lw + beta * J[e] * X[:, x] * X[:, x + 1]
    m = lw.max()
    v = torch.exp(lw - m)
    acc = m
    spin = torch.tensor([1.0, -1.0], dtype=DT)
    for y in range(1, Ly):
        for x in range(Lx):
            site = y * Lx + x
            ev = bond.get((site - Lx, site))
            Bv = torch.exp(beta * J[ev] * torch.outer(spin, spin)) if ev is not None else torch.ones(2, 2, dtype=DT)
            v3 = v.reshape(2 ** (Lx - 1 - x), 2, 2 ** x)
            v3 = torch.einsum("aoc,ot->atc", v3, Bv)
            if x > 0:
                eh = bond.get((site - 1, site))
                if eh is not None:
                    left = spin[(torch.arange(2 ** x) >> (x - 1)) & 1]  # bit x-1 of c
                    fac = torch.exp(beta * J[eh] * spin[:, None] * left[None, :])  # [t, c]
                    v3 = v3 * fac[None, :, :]
            v = v3.reshape(-1)
            m = v.max()
            v = v / m
            acc = acc + torch.log(m)
    return acc + torch.log(v.sum())


def kaufman_log_z(m: int, n: int, K: float) -> float:
    """Kaufman's exact ln Z for the ferromagnetic Ising model on an m x n torus
    (m rows, n spins per row) with coupling K = beta J > 0:
      Z = 1/2 (2 sinh 2K)^{mn/2} [ P_c(odd) + P_s(odd) + P_c(even) + P_s(even) ],
      P_c(set) = prod_{l in set} 2 cosh(m g_l / 2),  P_s(set) = prod 2 sinh(m g_l / 2),
      cosh g_l = cosh 2K coth 2K - cos(pi l / n), l = 0..2n-1,
    with g_0 = 2K + ln tanh K taken with its sign (it is negative above T_c,
    positive below)."""
    c = math.cosh(2 * K) / math.tanh(2 * K)
    g = []
    for l in range(2 * n):
        if l == 0:
            g.append(2 * K + math.log(math.tanh(K)))
        else:
            g.append(math.acosh(c - math.cos(math.pi * l / n)))
    odd = [g[l] for l in range(1, 2 * n, 2)]
    even = [g[l] for l in range(0, 2 * n, 2)]
    # Sum the four products in log space with signs.
    terms = []
    for gs in (odd, even):
        lc = sum(math.log(2 * math.cosh(m * x / 2)) for x in gs)
        terms.append((1.0, lc))
        sgn = 1.0
        ls = 0.0
        for x in gs:
            v = 2 * math.sinh(m * x / 2)
            if v == 0.0:
                sgn = 0.0
                break
            sgn *= math.copysign(1.0, v)
            ls += math.log(abs(v))
        if sgn != 0.0:
            terms.append((sgn, ls))
    mx = max(t[1] for t in terms)
    s = sum(sg * math.exp(l - mx) for sg, l in terms)
    return math.log(0.5) + 0.5 * m * n * math.log(2 * math.sinh(2 * K)) + mx + math.log(s)


def onsager_f(beta: float, J: float = 1.0, n_quad: int = 400) -> float:
    """Onsager's free energy per spin of the infinite square lattice:
    -beta f = ln 2 + 1/(8 pi^2) int_0^{2pi} int_0^{2pi}
              ln[cosh^2 2K - sinh 2K (cos t1 + cos t2)] dt1 dt2,  K = beta J,
    by the periodic trapezoid rule (exponentially convergent off T_c)."""
    K = beta * J
    t = np.arange(n_quad) * (2 * np.pi / n_quad)
    c1, c2 = np.meshgrid(np.cos(t), np.cos(t))
    integrand = np.log(np.cosh(2 * K) ** 2 - np.sinh(2 * K) * (c1 + c2))
    integral = integrand.mean() * (2 * np.pi) ** 2
    return -(math.log(2) + integral / (8 * math.pi ** 2)) / beta
