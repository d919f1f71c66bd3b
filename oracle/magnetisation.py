"""Magnetisation and susceptibility from samples (Sec. 3: once trained, the
network's samples give magnetisation and susceptibility), FP64.  Test
infrastructure only.

For one width-set configuration s, the leftover spins follow the Boltzmann
distribution conditional on s, p(r | s) ~ exp(-beta E(s, r)).  With a uniform
field h on R added to the energy (-h sum_{i in R} r_i), log Z_R(s; h) is the
cumulant generating function of M_R = sum_{i in R} r_i in the variable beta h:
  E[M_R | s]   = d log Z_R / d(beta h)       at h = 0,
  Var(M_R | s) = d^2 log Z_R / d(beta h)^2   at h = 0.
The total magnetisation M = M_W(s) + M_R therefore has E[M | s] = M_W(s) +
E[M_R | s] and Var(M | s) = Var(M_R | s).  Over samples s_b ~ q with
self-normalised importance weights w_b ~ exp(log Z_R(s_b) - log q(s_b)),
  <M>   = sum_b w_b E[M | s_b],
  <M^2> = sum_b w_b (E[M | s_b]^2 + Var(M | s_b)),
  chi   = beta (<M^2> - <M>^2) / N  (per spin).
"""
import torch

from .ising import DT


def conditional_moments(contract, sW: torch.Tensor, W, beta):
    """(E[M | s_b], Var(M | s_b)) for each row of sW [B, |W|], where
    contract(field) is log Z_R(s_b; field_b) ([B]) of any exact contraction
    with a per-sample uniform field on R.  Autograd twice: the rows are
    independent, so the gradient of the sum w.r.t. field_b is d/dfield_b of row b."""
    sW = torch.as_tensor(sW, dtype=DT)
    h = torch.zeros(sW.shape[0], dtype=DT, requires_grad=True)
    lz = contract(h)
    (g1,) = torch.autograd.grad(lz.sum(), h, create_graph=True)
    (g2,) = torch.autograd.grad(g1.sum(), h)
    mean = sW.sum(1) + g1.detach() / beta
    var = g2.detach() / (beta * beta)
    return mean, var


def magnetisation_stats(log_zr, logq, mean, var, beta, n):
    """(<M>, <M^2>, chi per spin, <M>_q, <M^2>_q, ESS) of one batch."""
    l = torch.as_tensor(log_zr, dtype=DT) - torch.as_tensor(logq, dtype=DT)
    w = torch.softmax(l, 0)
    mu = torch.as_tensor(mean, dtype=DT)
    m2 = mu * mu + torch.as_tensor(var, dtype=DT)
    M1, M2 = float((w * mu).sum()), float((w * m2).sum())
    return (M1, M2, beta * (M2 - M1 * M1) / n, float(mu.mean()), float(m2.mean()), float(1.0 / (w * w).sum()))
