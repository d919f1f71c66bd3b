"""Estimators of Sec. 3 in FP64.  Test infrastructure only.

With l_b = log Z_R(s_b) - log q(s_b) for samples s_b ~ q (this project's
reading: log Z_R includes -beta E_1, so Etilde = -log Z_R / beta):
  F_q      = -(1/beta) mean_b l_b                          (Eq. 9)
  log Z_IS = logsumexp_b l_b - ln B,  F_IS = -log Z_IS / beta
  stderr   = std_b(l_b) / (beta sqrt(B))  (sample std, ddof = 1)
  w_b      = -(l_b - mean l) / (beta B)      (Eq. 10 with the batch-mean baseline)
  grad     = sum_b w_b grad_theta log q(s_b)  (Eq. 10)
Exact (enumerated) F_q and its gradient over all 2^D width-set states pin the
sampled forms.  Adam follows Kingma & Ba (2015), Algorithm 1.
Observables (Sec. 3: samples of the trained network give Boltzmann averages):
self-normalised importance weights w_b = exp(l_b) / sum_b' exp(l_b') and the
exact conditional energy of a sample E_b = -d log Z_R(s_b) / d beta (Eq. 4)
give U = sum_b w_b E_b, its mean under q, and ESS = 1 / sum_b w_b^2.
"""
import math

import numpy as np
import torch

from . import made
from .ising import DT, all_configs


def free_energies(log_zr, logq, beta):
    l = torch.as_tensor(log_zr, dtype=DT) - torch.as_tensor(logq, dtype=DT)
    B = l.shape[0]
    fq = -l.mean() / beta
    lz = torch.logsumexp(l, 0) - math.log(B)
    se = (l.std(unbiased=True) / (beta * math.sqrt(B))) if B > 1 else torch.zeros((), dtype=DT)
    return {"F_q": float(fq), "F_IS": float(-lz / beta), "stderr": float(se), "logZ_IS": float(lz)}


def is_observables(log_zr, logq, energy):
    """(U, U_q, ESS) of one batch: energy = E_b = -d log Z_R(s_b) / d beta."""
    l = torch.as_tensor(log_zr, dtype=DT) - torch.as_tensor(logq, dtype=DT)
    w = torch.softmax(l, 0)
    E = torch.as_tensor(energy, dtype=DT)
    return float((w * E).sum()), float(E.mean()), float(1.0 / (w * w).sum())


def reinforce_weights(log_zr, logq, beta):
    l = torch.as_tensor(log_zr, dtype=DT) - torch.as_tensor(logq, dtype=DT)
    return -(l - l.mean()) / (beta * l.shape[0])


def surrogate_grad(theta, D, hidden, s, w):
    """grad_theta of sum_b w_b log q_theta(s_b), w held fixed (torch autograd)."""
    th = torch.as_tensor(theta, dtype=DT).clone().requires_grad_(True)
    obj = (torch.as_tensor(w, dtype=DT) * made.log_q(th, D, hidden, torch.as_tensor(s, dtype=DT))).sum()
    (g,) = torch.autograd.grad(obj, th)
    return g


def exact_fq(theta, D, hidden, log_zr_all, beta):
    """F_q = sum_s q(s) [-(log Z_R(s) - log q(s)) / beta] over all 2^D states
    (rows ordered as ising.all_configs(D))."""
    lq = made.all_log_q(torch.as_tensor(theta, dtype=DT), D, hidden)
    return (torch.exp(lq) * (-(torch.as_tensor(log_zr_all, dtype=DT) - lq) / beta)).sum()


def exact_grad(theta, D, hidden, log_zr_all, beta):
    """Eq. 10 evaluated exactly: sum_s q(s) f(s) grad log q(s), f = -(log Z_R - log q)/beta."""
    th = torch.as_tensor(theta, dtype=DT).clone().requires_grad_(True)
    X = all_configs(D)
    lq = made.log_q(th, D, hidden, X)
    f = (-(torch.as_tensor(log_zr_all, dtype=DT) - lq) / beta).detach()
    q = torch.exp(lq).detach()
    (g,) = torch.autograd.grad((q * f * lq).sum(), th)
    return g


def adam_step(p, g, m, v, t, lr=0.01, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t >= 1 is the step count after this update)."""
    p, g, m, v = (np.asarray(x, np.float64) for x in (p, g, m, v))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
