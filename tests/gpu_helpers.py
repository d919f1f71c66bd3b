"""Shared helpers for the GPU parity tests: oracle replay of the sampler and
upload of oracle-drawn configurations (inputs always flow oracle -> GPU)."""
import numpy as np
import torch

from oracle import made, philox


def oracle_samples(params_f32: np.ndarray, D: int, hidden, seed: int, step: int, instance: int, batch: int,
                   rows=None):
    """Replay Eq. 8 in FP64 with the same Philox uniforms; rows = sample indices."""
    theta = torch.as_tensor(np.asarray(params_f32, np.float64))
    u = philox.uniforms(seed, step, instance, batch, D)
    if rows is not None:
        u = u[rows]
    s, p = made.sample(theta, D, hidden, u)
    return s, p, u


def check_sample_agreement(s_gpu: np.ndarray, s_or: np.ndarray, u: np.ndarray, p_or: np.ndarray,
                           max_flip_frac: float = 2e-3, window: float = 1e-5):
    """Samples are not unique across precisions: every row must match the
    oracle's draw except rows whose first disagreement sits where u is within
    `window` of the oracle's FP64 probability (a legitimate rounding flip)."""
    diff = np.any(s_gpu != s_or, axis=1)
    for b in np.flatnonzero(diff):
        i = int(np.flatnonzero(s_gpu[b] != s_or[b])[0])
        assert abs(u[b, i] - p_or[b, i]) < window, (b, i, u[b, i], p_or[b, i])
    assert diff.mean() <= max_flip_frac
    return ~diff


def to_dev_spins(s: np.ndarray) -> torch.Tensor:
    return torch.as_tensor(np.asarray(s, np.int8).reshape(-1)).cuda()
