"""MADE autoregressive network in FP64 (Eq. 6-8; Fig. 1(d) cites MADE,
Germain et al. 2015).  Test infrastructure only.

Architecture (the paper's Eq. 7 is one masked layer; hidden layers follow MADE):
  * inputs/outputs i = 0..D-1 carry degree i+1 (the autoregressive order);
  * hidden unit k of every hidden layer carries degree m(k) = (k mod max(D-1,1)) + 1;
  * masks: input j -> hidden k iff m(k) >= j+1; hidden k -> next hidden k'
    iff m(k') >= m(k); last hidden k -> output i iff i+1 > m(k); with no hidden
    layer, input j -> output i iff i > j;
  * ReLU between layers, logit x_i at the output, q(s_i=+1|s_<i) = sigmoid(x_i);
  * unsampled inputs are 0 (the masks make them irrelevant).
Flat parameter layout, layer by layer: W_l [out][in] row-major, then b_l [out].
  log q(s) = sum_i log q(s_i|s_<i) = sum_i -softplus(-s_i x_i)            (Eq. 6, 8)
"""
import numpy as np
import torch
import torch.nn.functional as F

from .ising import DT, all_configs


def layer_sizes(D, hidden):
    return [D] + list(hidden) + [D]


def n_params(D, hidden):
    sz = layer_sizes(D, hidden)
    return sum(sz[l + 1] * sz[l] + sz[l + 1] for l in range(len(sz) - 1))


def degrees(D, hidden):
    """Degree vectors per layer (inputs, hidden..., outputs)."""
    cyc = max(D - 1, 1)
    degs = [np.arange(1, D + 1)]
    for H in hidden:
        degs.append(np.arange(H) % cyc + 1)
    degs.append(np.arange(1, D + 1))
    return degs


def masks(D, hidden):
    """List of [out, in] 0/1 masks."""
    degs = degrees(D, hidden)
    out = []
    L = len(degs) - 1
    for l in range(L):
        din, dout = degs[l], degs[l + 1]
        if l == L - 1:
            m = dout[:, None] > din[None, :]
        else:
            m = dout[:, None] >= din[None, :]
        out.append(torch.as_tensor(m.astype(np.float64)))
    return out


def unpack(theta: torch.Tensor, D, hidden):
    sz = layer_sizes(D, hidden)
    layers = []
    off = 0
    for l in range(len(sz) - 1):
        nin, nout = sz[l], sz[l + 1]
        Wl = theta[off:off + nout * nin].reshape(nout, nin)
        off += nout * nin
        bl = theta[off:off + nout]
        off += nout
        layers.append((Wl, bl))
    assert off == theta.numel()
    return layers


def logits(theta: torch.Tensor, D, hidden, s: torch.Tensor) -> torch.Tensor:
    """x [B, D] for inputs s [B, D] (+-1, or 0 where unsampled)."""
    theta = theta.to(DT)
    layers = unpack(theta, D, hidden)
    ms = masks(D, hidden)
    h = s.to(DT)
    for l, ((Wl, bl), ml) in enumerate(zip(layers, ms)):
        h = h @ (Wl * ml).T + bl
        if l < len(layers) - 1:
            h = torch.relu(h)
    return h


def log_q(theta, D, hidden, s: torch.Tensor) -> torch.Tensor:
    """log q(s) for complete samples s [B, D] of +-1 (Eq. 6 and 8)."""
    x = logits(theta, D, hidden, s)
    return -F.softplus(-s.to(DT) * x).sum(1)


def sample(theta, D, hidden, u: np.ndarray):
    """Ancestral sampling (Eq. 8, Sec. 3): for i = 1..D, run the network on the
    spins drawn so far, p_i = sigmoid(x_i), s_i = +1 iff u[:, i] < p_i.
    Returns (s [B, D] float64, p [B, D] the conditional probabilities used)."""
    u = torch.as_tensor(u, dtype=DT)
    B = u.shape[0]
    s = torch.zeros(B, D, dtype=DT)
    p = torch.zeros(B, D, dtype=DT)
    with torch.no_grad():
        for i in range(D):
            x = logits(theta, D, hidden, s)[:, i]
            p[:, i] = torch.sigmoid(x)
            s[:, i] = torch.where(u[:, i] < p[:, i], 1.0, -1.0)
    return s, p


def all_log_q(theta, D, hidden) -> torch.Tensor:
    """log q over all 2^D configurations (rows of ising.all_configs(D))."""
    return log_q(theta, D, hidden, all_configs(D))


def init_params(D, hidden, seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (PyTorch's
    default Linear initialisation), flat layout, float64."""
    rng = np.random.default_rng(seed)
    sz = layer_sizes(D, hidden)
    parts = []
    for l in range(len(sz) - 1):
        bound = 1.0 / np.sqrt(sz[l])
        parts.append(rng.uniform(-bound, bound, size=sz[l + 1] * sz[l]))
        parts.append(rng.uniform(-bound, bound, size=sz[l + 1]))
    return np.concatenate(parts)
