"""Eq. 4 for general leftover components (random-graph workload), FP64.
Test infrastructure only.

Each connected component c of the graph on R contributes
  ln Z_c(s) = ln sum_{r_c} prod_{(i,j) in c} exp(beta J_ij r_i r_j)
                           prod_{i in c} exp(beta h_i(s) r_i),
  h_i(s) = sum_{k in W, k~i} J_ik s_k,
computed either by enumerating r_c (|c| <= `enum_max`) or by variable
elimination in a minimum-degree order (the order is the oracle's own: at each
step the variable with the fewest neighbours, ties to the lowest index, or with
order_rule="min_degree_high" to the highest index, a second route for
cross-checks).
"""
import numpy as np
import torch

from .ising import DT, all_configs, components, w_energy_term

_SPIN = torch.tensor([1.0, -1.0], dtype=DT)


def _fields(ei, ej, J, W, sW, comp):
    """h[b, k] for the spins of comp (in comp order)."""
    wpos = {int(w): k for k, w in enumerate(np.asarray(W).tolist())}
    cpos = {v: k for k, v in enumerate(comp)}
    h = torch.zeros(sW.shape[0], len(comp), dtype=DT)
    for e, (a, b) in enumerate(zip(np.asarray(ei).tolist(), np.asarray(ej).tolist())):
        if a in cpos and b in wpos:
            h[:, cpos[a]] = h[:, cpos[a]] + J[e] * sW[:, wpos[b]]
        elif b in cpos and a in wpos:
            h[:, cpos[b]] = h[:, cpos[b]] + J[e] * sW[:, wpos[a]]
    return h


def _inner_edges(ei, ej, comp):
    cpos = {v: k for k, v in enumerate(comp)}
    out = []
    for e, (a, b) in enumerate(zip(np.asarray(ei).tolist(), np.asarray(ej).tolist())):
        if a in cpos and b in cpos:
            out.append((e, cpos[a], cpos[b]))
    return out


def _comp_enum(J, beta, comp, inner, h):
    X = all_configs(len(comp))  # [S, k]
    expo = beta * (h @ X.T)  # [B, S]
    for e, a, b in inner:
        expo = expo + (beta * J[e] * X[:, a] * X[:, b])[None, :]
    return torch.logsumexp(expo, dim=1)


def _comp_elim(J, beta, comp, inner, h, order=None, order_rule="min_degree"):
    """Variable elimination on factor tables with a batch axis.  A factor is
    (list of variables, tensor [B, 2, ..., 2]); index 0 = spin +1."""
    B = h.shape[0]
    factors = []
    for k in range(len(comp)):
        factors.append(([k], torch.exp(beta * h[:, k:k + 1] * _SPIN[None, :])))
    for e, a, b in inner:
        t = torch.exp(beta * J[e] * torch.outer(_SPIN, _SPIN))
        factors.append(([a, b], t[None].expand(B, 2, 2)))
    logacc = torch.zeros(B, dtype=DT)
    remaining = set(range(len(comp)))
    # neighbours of each variable: the other variables it shares a factor with
    # (the bonds, then the scopes of the tables created so far)
    nbrs = {k: set() for k in range(len(comp))}
    for e, a, b in inner:
        nbrs[a].add(b)
        nbrs[b].add(a)
    while remaining:
        if order is None:
            cand = sorted(remaining, reverse=(order_rule == "min_degree_high"))
            v = min(cand, key=lambda u: len(nbrs[u]))
        else:
            v = next(u for u in order if u in remaining)
        remaining.discard(v)
        for a in nbrs[v]:
            nbrs[a] |= nbrs[v]
            nbrs[a].discard(a)
            nbrs[a].discard(v)
        del nbrs[v]
        use = [f for f in factors if v in f[0]]
        factors = [f for f in factors if v not in f[0]]
        vars_out = sorted(set(x for vs, _ in use for x in vs) - {v})
        allv = vars_out + [v]
        letters = "abcdefghijklmnopqrstuvwxyz"
        if len(allv) > 20:
            raise ValueError("elimination width too large for the oracle")
        spec = ",".join("Z" + "".join(letters[allv.index(x)] for x in vs) for vs, _ in use)
        spec += "->Z" + "".join(letters[allv.index(x)] for x in vars_out)
        t = torch.einsum(spec, *[tt for _, tt in use])
        m = t.reshape(B, -1).max(dim=1).values
        t = t / m.reshape([B] + [1] * len(vars_out))
        logacc = logacc + torch.log(m)
        factors.append((vars_out, t))
    for vs, t in factors:  # all remaining factors are scalars per sample
        logacc = logacc + torch.log(t.reshape(B))
    return logacc


def log_zr_general(n, ei, ej, J, beta, W, sW: torch.Tensor, enum_max: int = 16,
                   order_rule: str = "min_degree", field=None) -> torch.Tensor:
    """-beta E_1(s) + sum_c ln Z_c(s) for each row of sW [B, |W|].  `field`
    ([B] or a scalar): a uniform field on R, added to every R spin's field."""
    J = torch.as_tensor(J, dtype=DT) if not torch.is_tensor(J) else J
    sW = sW.to(DT)
    total = w_energy_term(ei, ej, J, beta, W, sW)
    for comp in components(n, ei, ej, W):
        inner = _inner_edges(ei, ej, comp)
        h = _fields(ei, ej, J, W, sW, comp)
        if field is not None:
            h = h + (field[:, None] if torch.is_tensor(field) and field.dim() > 0 else field)
        if len(comp) <= enum_max:
            total = total + _comp_enum(J, beta, comp, inner, h)
        else:
            total = total + _comp_elim(J, beta, comp, inner, h, None, order_rule)
    return total
