"""Ising energy, brute-force partition function and per-sample log Z_R by
plain enumeration (FP64).  Test infrastructure only.

Conventions (Sec. 2):
  E(s) = - sum_<ij> J_ij s_i s_j,  p(s) = exp(-beta E)/Z,  F = -ln Z / beta  (Eq. 1-2)
  Z = sum_{s in W} sum_{r in R} exp(-beta E(s, r)) = sum_{s in W} exp(-beta Etilde(s))  (Eq. 3)
  Etilde(s) = E_1(s) - (1/beta) ln sum_r exp(-beta E_2(s, r))                 (Eq. 4)
This project's per-sample quantity is log Z_R(s) := -beta Etilde(s), i.e. it
includes the W-W term -beta E_1(s).  Since E(s, r) = E_1(s) + E_2(s, r), it
equals ln sum_r exp(-beta E(s, r)), which is what `log_zr_enum` sums.
"""
import numpy as np
import torch

DT = torch.float64


def all_configs(n: int) -> torch.Tensor:
    """All 2^n configurations as a [2^n, n] +/-1 tensor; bit k of the row
    index set means spin k = -1."""
    idx = torch.arange(2 ** n, dtype=torch.int64)[:, None]
    bits = (idx >> torch.arange(n, dtype=torch.int64)[None, :]) & 1
    return (1 - 2 * bits).to(DT)


def energy(ei, ej, J, s: torch.Tensor) -> torch.Tensor:
    """E(s) = -sum_<ij> J_ij s_i s_j (Eq. 1) for s of shape [..., n]."""
    ei = torch.as_tensor(np.asarray(ei), dtype=torch.int64)
    ej = torch.as_tensor(np.asarray(ej), dtype=torch.int64)
    J = torch.as_tensor(J, dtype=DT)
    return -(J * s[..., ei] * s[..., ej]).sum(-1)


def log_z_brute(n: int, ei, ej, J, beta) -> torch.Tensor:
    """ln Z = ln sum_s exp(-beta E(s)) over all 2^n states (Eq. 2), n <= 22.
    `J` and `beta` may be tensors requiring grad."""
    total = None
    chunk = 1 << min(n, 16)
    for start in range(0, 2 ** n, chunk):
        idx = torch.arange(start, min(start + chunk, 2 ** n), dtype=torch.int64)[:, None]
        s = (1 - 2 * ((idx >> torch.arange(n)[None, :]) & 1)).to(DT)
        part = torch.logsumexp(-beta * energy(ei, ej, J, s), dim=0)
        total = part if total is None else torch.logaddexp(total, part)
    return total


def log_zr_enum(n: int, ei, ej, J, beta, W, sW: torch.Tensor, field=None) -> torch.Tensor:
    """log Z_R(s) = ln sum_{r in {+-1}^|R|} exp(-beta E(s, r)) for each row s
    of sW [B, |W|] (Eq. 3-4 with E_1 included), by enumerating R (|R| <= 20).
    With `field` ([B] or a scalar), a uniform field on the R spins adds
    beta * field * sum_{i in R} r_i to every exponent (its derivatives at 0
    give the magnetisation moments of R)."""
    W = np.asarray(W, np.int64)
    R = np.setdiff1d(np.arange(n), W)
    rc = all_configs(len(R))  # [2^|R|, |R|]
    out = []
    for b in range(sW.shape[0]):
        full = torch.zeros(rc.shape[0], n, dtype=DT)
        full[:, torch.as_tensor(R)] = rc
        full[:, torch.as_tensor(W)] = sW[b].to(DT)[None, :]
        expo = -beta * energy(ei, ej, J, full)
        if field is not None:
            hb = field[b] if torch.is_tensor(field) and field.dim() > 0 else field
            expo = expo + beta * hb * rc.sum(1)
        out.append(torch.logsumexp(expo, dim=0))
    return torch.stack(out)


def components(n: int, ei, ej, W):
    """Connected components of the graph induced on R = all spins not in W,
    each a sorted list of spin indices (breadth-first search)."""
    Wset = set(int(w) for w in np.asarray(W).tolist())
    adj = [[] for _ in range(n)]
    for a, b in zip(np.asarray(ei).tolist(), np.asarray(ej).tolist()):
        adj[a].append(b)
        adj[b].append(a)
    seen = set(Wset)
    comps = []
    for v in range(n):
        if v in seen:
            continue
        queue = [v]
        seen.add(v)
        k = 0
        while k < len(queue):
            u = queue[k]
            k += 1
            for w in adj[u]:
                if w not in seen:
                    seen.add(w)
                    queue.append(w)
        comps.append(sorted(queue))
    return comps


def w_energy_term(ei, ej, J, beta, W, sW: torch.Tensor) -> torch.Tensor:
    """-beta E_1(s): the W-W bonds only (Eq. 4), for sW [B, |W|]."""
    pos = {int(w): k for k, w in enumerate(np.asarray(W).tolist())}
    J = torch.as_tensor(J, dtype=DT)
    tot = torch.zeros(sW.shape[0], dtype=DT)
    for e, (a, b) in enumerate(zip(np.asarray(ei).tolist(), np.asarray(ej).tolist())):
        if a in pos and b in pos:
            tot = tot + beta * J[e] * sW[:, pos[a]].to(DT) * sW[:, pos[b]].to(DT)
    return tot
