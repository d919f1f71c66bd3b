"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written from the published definition.

Used to reproduce the uniforms u_{b,i} behind the Bernoulli draw of Eq. 8
(s_i = +1 iff u_{b,i} < q(s_i=+1|s_<i)).  Counter and key conventions of this
project:
    counter = (b, i >> 2, step mod 2^32, instance),  key = (seed mod 2^32, seed >> 32)
    word    = output[i & 3],   u = (word >> 8) * 2^-24   (24-bit uniform in [0, 1)).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint array [..., 4], key: uint array [..., 2] (values < 2^32).
    Returns uint64 array [..., 4] of 32-bit words."""
    c = [np.asarray(ctr[..., j], np.uint64) & _MASK for j in range(4)]
    k0 = np.asarray(key[..., 0], np.uint64) & _MASK
    k1 = np.asarray(key[..., 1], np.uint64) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c[0]  # < 2^64, exact in uint64
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def uniforms(seed: int, step: int, instance: int, batch: int, D: int) -> np.ndarray:
    """u[b, i] for b < batch, i < D as float64 (exact 24-bit values)."""
    b = np.arange(batch, dtype=np.uint64)[:, None]
    i = np.arange(D, dtype=np.uint64)[None, :]
    shape = (batch, D)
    ctr = np.stack([np.broadcast_to(b, shape),
                    np.broadcast_to(i >> np.uint64(2), shape),
                    np.full(shape, step & 0xFFFFFFFF, np.uint64),
                    np.full(shape, instance & 0xFFFFFFFF, np.uint64)], axis=-1)
    key = np.stack([np.full(shape, seed & 0xFFFFFFFF, np.uint64),
                    np.full(shape, (seed >> 32) & 0xFFFFFFFF, np.uint64)], axis=-1)
    out = philox4x32_10(ctr, key)
    word = np.take_along_axis(out, (np.broadcast_to(i, shape) & np.uint64(3)).astype(np.int64)[..., None],
                              axis=-1)[..., 0]
    return (word >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
