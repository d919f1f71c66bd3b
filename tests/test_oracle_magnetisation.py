"""Pins of oracle/magnetisation.py (Sec. 3: magnetisation and susceptibility
from samples) against what the mathematics fixes: the conditional moments by
plain enumeration of p(r | s), closed forms (independent spins in a field, the
open chain in zero field), agreement of the independent contraction routes,
and, with a census of every width-set state under a uniform q, the exact
Boltzmann moments of the whole system by brute force."""
import math

import numpy as np
import torch

from oracle import dense, general, ising, transfer
from oracle import magnetisation as mg

DT = torch.float64


def _random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    pairs = set()
    while len(pairs) < m:
        a, b = sorted(rng.choice(n, 2, replace=False).tolist())
        pairs.add((a, b))
    ei, ej = zip(*sorted(pairs))
    return np.array(ei), np.array(ej), rng.normal(0.0, 1.0, size=m)


def _enumerated_moments(n, ei, ej, J, beta, W, sW):
    """E[M | s] and Var(M | s) straight from p(r | s) ~ exp(-beta E(s, r))."""
    R = [v for v in range(n) if v not in set(W)]
    mean, var = [], []
    for s in sW:
        ws, ms = [], []
        for idx in range(2 ** len(R)):
            full = np.zeros(n)
            full[list(W)] = s
            for k, v in enumerate(R):
                full[v] = -1.0 if (idx >> k) & 1 else 1.0
            E = -sum(J[e] * full[ei[e]] * full[ej[e]] for e in range(len(ei)))
            ws.append(math.exp(-beta * E))
            ms.append(full.sum())
        ws, ms = np.array(ws) / sum(ws), np.array(ms)
        mu = float((ws * ms).sum())
        mean.append(mu)
        var.append(float((ws * (ms - mu) ** 2).sum()))
    return np.array(mean), np.array(var)


def test_moments_equal_the_enumerated_definition():
    n, beta = 10, 0.8
    ei, ej, J = _random_graph(n, 18, 3)
    W = [1, 4, 7]
    rng = np.random.default_rng(4)
    sW = np.where(rng.random((6, 3)) < 0.5, 1.0, -1.0)
    ref_m, ref_v = _enumerated_moments(n, ei, ej, J, beta, W, sW)
    st = torch.as_tensor(sW)
    for contract in (lambda h: ising.log_zr_enum(n, ei, ej, J, beta, W, st, field=h),
                     lambda h: dense.log_zr_dense(n, ei, ej, J, beta, W, st, field=h),
                     lambda h: general.log_zr_general(n, ei, ej, J, beta, W, st, field=h),
                     lambda h: general.log_zr_general(n, ei, ej, J, beta, W, st, enum_max=0, field=h)):
        m, v = mg.conditional_moments(contract, st, W, beta)
        assert np.allclose(m.numpy(), ref_m, rtol=0, atol=1e-10)
        assert np.allclose(v.numpy(), ref_v, rtol=0, atol=1e-10)


def test_independent_spins_in_a_field():
    # every R spin bonded only to width-set spins: independent given s, so
    # E[M_R | s] = sum tanh(beta h_i), Var = sum sech^2(beta h_i)
    W = [0, 1]
    R = list(range(2, 8))
    rng = np.random.default_rng(5)
    ei, ej, J = [], [], []
    for r in R:
        for w in W:
            ei.append(w)
            ej.append(r)
            J.append(rng.normal())
    ei, ej, J = np.array(ei), np.array(ej), np.array(J)
    ei, ej, J = np.append(ei, 0), np.append(ej, 1), np.append(J, 0.7)  # a W-W bond changes nothing
    beta, n = 1.3, 8
    sW = torch.tensor([[1.0, 1.0], [1.0, -1.0], [-1.0, -1.0]], dtype=DT)
    for contract in (lambda h: general.log_zr_general(n, ei, ej, J, beta, W, sW, enum_max=0, field=h),
                     lambda h: dense.log_zr_dense(n, ei, ej, J, beta, W, sW, field=h)):
        m, v = mg.conditional_moments(contract, sW, W, beta)
        for b in range(3):
            h = np.array([sum(J[e] * float(sW[b, W.index(ei[e])]) for e in range(len(R) * 2) if ej[e] == r)
                          for r in R])
            assert abs(float(m[b]) - (float(sW[b].sum()) + np.tanh(beta * h).sum())) <= 1e-12
            assert abs(float(v[b]) - (1.0 / np.cosh(beta * h) ** 2).sum()) <= 1e-12


def test_open_chain_in_zero_field():
    # a 2 x L lattice, W = column 0, the bonds between the columns zero: the R
    # column is an open chain in zero field, <r_i r_j> = prod of tanh(beta J_k)
    # between i and j, so E[M_R] = 0 and Var(M_R) = sum_{i,j} prod_k t_k
    L, beta = 9, 0.9
    rng = np.random.default_rng(6)
    ei, ej, J = [], [], []
    Jv = rng.normal(0.0, 1.2, size=L - 1)
    for y in range(L):
        ei.append(2 * y)
        ej.append(2 * y + 1)
        J.append(0.0)
        if y + 1 < L:
            ei += [2 * y, 2 * y + 1]
            ej += [2 * y + 2, 2 * y + 3]
            J += [rng.normal(), Jv[y]]
    ei, ej, J = np.array(ei), np.array(ej), np.array(J)
    W = [2 * y for y in range(L)]
    t = np.tanh(beta * Jv)
    var_ref = sum(np.prod(t[min(i, j):max(i, j)]) for i in range(L) for j in range(L))
    sW = torch.as_tensor(np.where(rng.random((4, L)) < 0.5, 1.0, -1.0))
    for contract in (lambda h: transfer.log_zr_lattice(2 * L, ei, ej, J, beta, W, sW, 2, field=h),
                     lambda h: general.log_zr_general(2 * L, ei, ej, J, beta, W, sW, enum_max=0, field=h)):
        m, v = mg.conditional_moments(contract, sW, W, beta)
        assert np.allclose(m.numpy(), sW.sum(1).numpy(), rtol=0, atol=1e-12)
        assert np.allclose(v.numpy(), var_ref, rtol=1e-12, atol=0)


def test_lattice_routes_agree():
    # two strips of width 2 on a 5 x 4 lattice: transfer matrices, plain
    # enumeration and elimination give the same moments
    Lx, Ly, beta = 5, 4, 0.6
    rng = np.random.default_rng(7)
    ei, ej = [], []
    for y in range(Ly):
        for x in range(Lx):
            v = y * Lx + x
            if x + 1 < Lx:
                ei.append(v)
                ej.append(v + 1)
            if y + 1 < Ly:
                ei.append(v)
                ej.append(v + Lx)
    ei, ej = np.array(ei), np.array(ej)
    J = rng.normal(size=len(ei))
    W = [y * Lx + x for y in range(Ly) for x in (2,)]
    n = Lx * Ly
    sW = torch.as_tensor(np.where(rng.random((5, len(W))) < 0.5, 1.0, -1.0))
    res = []
    for contract in (lambda h: transfer.log_zr_lattice(n, ei, ej, J, beta, W, sW, Lx, field=h),
                     lambda h: ising.log_zr_enum(n, ei, ej, J, beta, W, sW, field=h),
                     lambda h: general.log_zr_general(n, ei, ej, J, beta, W, sW, enum_max=0, field=h)):
        res.append(mg.conditional_moments(contract, sW, W, beta))
    for m, v in res[1:]:
        assert torch.allclose(m, res[0][0], rtol=0, atol=1e-10)
        assert torch.allclose(v, res[0][1], rtol=0, atol=1e-10)


def test_census_gives_the_boltzmann_moments():
    # every width-set state once under a uniform q: the importance weights are
    # then the exact marginal p(s), and <M>, <M^2> the exact Boltzmann moments
    n, beta = 11, 0.7
    ei, ej, J = _random_graph(n, 20, 8)
    J = J + 0.5  # mostly ferromagnetic
    W = [0, 3, 5, 9]
    sW = ising.all_configs(len(W))
    lz = ising.log_zr_enum(n, ei, ej, J, beta, W, sW)
    lq = torch.full((sW.shape[0],), -len(W) * math.log(2.0), dtype=DT)
    m, v = mg.conditional_moments(lambda h: ising.log_zr_enum(n, ei, ej, J, beta, W, sW, field=h), sW, W, beta)
    M1, M2, chi, M1q, M2q, ess = mg.magnetisation_stats(lz, lq, m, v, beta, n)
    X = ising.all_configs(n)
    p = torch.softmax(-beta * ising.energy(ei, ej, J, X), 0)
    M = X.sum(1)
    ref1, ref2 = float((p * M).sum()), float((p * M * M).sum())
    assert abs(M1 - ref1) <= 1e-10  # 0 by the spin-flip symmetry
    assert abs(ref1) <= 1e-10
    assert abs(M2 - ref2) <= 1e-10 * ref2
    assert abs(chi - beta * (ref2 - ref1 ** 2) / n) <= 1e-10 * ref2
    # under q: the uniform average over s of the conditional moments
    assert abs(M1q - float(m.mean())) <= 1e-12 and abs(M2q - float((m * m + v).mean())) <= 1e-12
    assert 1.0 <= ess <= sW.shape[0]
    # equal weights: ESS = B
    assert abs(mg.magnetisation_stats(lz, lz, m, v, beta, n)[5] - sW.shape[0]) <= 1e-9
