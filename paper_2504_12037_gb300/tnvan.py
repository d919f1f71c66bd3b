"""Thin ctypes binding of libtnvan.so (the C-ABI in include/tnvan.h).

The functions here only marshal arguments: every step of the hot path runs in
the library's CUDA kernels.  Tensors are torch CUDA tensors (device memory and
streams only); host arrays are NumPy.  There is no CPU fallback: if the library
is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtnvan.so")

OK = 0
E_ARG, E_NOMEM, E_CUDA, E_TIMEOUT, E_OVERFLOW, E_STATE, E_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
LATTICE2D, DENSE, GENERAL = 0, 1, 2
FP32, TF32, BF16 = 0, 1, 2
SLICE_FIXED, SLICE_GREEDY, SLICE_BEST = 1, 2, 3

_c_int, _c_i64, _c_u64, _c_dbl, _vp = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_dblp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); mirrors include/tnvan.h
SIGNATURES = {
    "tnvan_version": (_c_int, []),
    "tnvan_create": (_c_int, [ctypes.POINTER(_vp), _c_int]),
    "tnvan_destroy": (_c_int, [_vp]),
    "tnvan_last_error": (ctypes.c_char_p, [_vp]),
    "tnvan_init_graph": (_c_int, [_vp, _c_int, _c_int, _c_int, _i32p, _i32p, _dblp, _c_int, _c_int, _c_int, _c_int]),
    "tnvan_set_width_set": (_c_int, [_vp, _c_int, _c_int, _i32p]),
    "tnvan_set_width_set_ordered": (_c_int, [_vp, _c_int, _c_int, _i32p, _i32p]),
    "tnvan_find_width_set": (_c_int, [_c_int, _c_int, _i32p, _i32p, _c_int, _c_int, _c_u64, _c_int, _c_int, _i32p,
                                      _i32p, _i32p]),
    "tnvan_set_made": (_c_int, [_vp, _c_int, _c_int, _i32p, _vp]),
    "tnvan_n_params": (_c_int, [_vp, _c_int, _i64p, _i64p]),
    "tnvan_instance_info": (_c_int, [_vp, _c_int, _i32p]),
    "tnvan_reserve": (_c_int, [_vp, _c_int]),
    "tnvan_sample_and_contract": (_c_int, [_vp, _dblp, _c_int, _c_u64, _c_u64, _c_int, _vp, _vp, _vp, _vp]),
    "tnvan_sample_contract_adjoint": (_c_int, [_vp, _dblp, _c_int, _c_u64, _c_u64, _c_int, _vp, _vp, _vp, _vp,
                                               _vp, _vp]),
    "tnvan_train_step": (_c_int, [_vp, _dblp, _c_int, _c_u64, _c_u64, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                  _vp, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_i64, _vp]),
    "tnvan_observables": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _vp, _vp, _dblp, _vp]),
    "tnvan_magnetisation": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _vp, _vp, _vp, _dblp, _vp]),
    "tnvan_log_prob": (_c_int, [_vp, _c_int, _vp, _c_int, _vp, _vp]),
    "tnvan_contract": (_c_int, [_vp, _dblp, _c_int, _vp, _c_int, _vp, _vp, _vp]),
    "tnvan_free_energy": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _dblp, _vp]),
    "tnvan_reduce": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _vp, _vp]),
    "tnvan_step_stats": (_c_int, [_vp, _vp, _vp]),
    "tnvan_merge_stats": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _vp]),
    "tnvan_backward_stats": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _vp, _c_int, _vp, _vp]),
    "tnvan_backward": (_c_int, [_vp, _dblp, _c_int, _vp, _vp, _vp, _c_int, _vp, _vp, _vp, _vp]),
    "tnvan_adam": (_c_int, [_vp, _c_i64, _vp, _vp, _vp, _vp, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_i64, _vp]),
    "tnvan_free_energy_noalloc": (_c_int, [_c_int, _c_int, _dblp, _vp, _vp, _vp, _vp]),
    "tnvan_noalloc_last_error": (ctypes.c_char_p, []),
    "tnvan_set_step_counter": (_c_int, [_vp, _vp]),
    "tnvan_autotune": (_c_int, [_vp, _dblp, _c_int, _c_int, _vp, _i32p]),
    "tnvan_set_tuning": (_c_int, [_vp, _i32p]),
    "tnvan_profile": (_c_int, [_vp, _c_int]),
    "tnvan_profile_read": (_c_int, [_vp, _c_int, ctypes.c_char_p, _c_int, _dblp, _i64p]),
    "tnvan_profile_trace": (_c_int, [_vp, ctypes.c_int64, _vp, _vp, _vp, _i64p]),
}

_LIB = None


class TnvanError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tnvan error {code}: {msg}")
        self.code = code


def lib():
    """Load libtnvan.so (built in-tree by build.py); raise if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    ctype = {np.int32: ctypes.c_int32, np.float64: ctypes.c_double, np.int64: ctypes.c_int64}[dtype]
    return a, a.ctypes.data_as(ctypes.POINTER(ctype))


def find_width_set(n_spins: int, ei, ej, w_u: int, restarts: int = 4, seed: int = 0, mode: int = SLICE_BEST,
                   anneal: int = 0):
    """Width-set finder (tnvan_find_width_set): returns (W, R's elimination
    order, achieved width, winning trial); `anneal` annealing moves refine the
    winner.  Host only."""
    ei, pi = _arr(ei, np.int32)
    ej, pj = _arr(ej, np.int32)
    out_w = np.zeros(n_spins, np.int32)
    out_o = np.zeros(n_spins, np.int32)
    info = np.zeros(3, np.int32)
    rc = lib().tnvan_find_width_set(n_spins, ei.shape[0], pi, pj, w_u, restarts, seed, mode, anneal,
                                    out_w.ctypes.data_as(_i32p), out_o.ctypes.data_as(_i32p),
                                    info.ctypes.data_as(_i32p))
    if rc != OK:
        raise TnvanError(rc, "tnvan_find_width_set: invalid argument")
    nw = int(info[0])
    return out_w[:nw].copy(), out_o[:n_spins - nw].copy(), int(info[1]), int(info[2])


class Context:
    """Owns one tnvan_ctx.  Method names follow the C-ABI."""

    def __init__(self, device: int = 0):
        self._h = _vp()
        rc = lib().tnvan_create(ctypes.byref(self._h), device)
        if rc != OK:
            raise TnvanError(rc, lib().tnvan_last_error(None).decode())
        self.device = device

    def _check(self, rc: int):
        if rc != OK:
            raise TnvanError(rc, lib().tnvan_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().tnvan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- set-up -----------------------------------------------------------
    def init_graph(self, instance: int, n_spins: int, ei, ej, J, topology: int, Lx: int = 0, Ly: int = 0,
                   periodic: bool = False):
        ei, pi = _arr(ei, np.int32)
        ej, pj = _arr(ej, np.int32)
        J, pJ = _arr(J, np.float64)
        self._check(lib().tnvan_init_graph(self._h, instance, n_spins, ei.shape[0], pi, pj, pJ, topology,
                                           Lx, Ly, int(periodic)))

    def set_width_set(self, instance: int, w, r_order=None):
        w, pw = _arr(w, np.int32)
        if r_order is None:
            self._check(lib().tnvan_set_width_set(self._h, instance, w.shape[0], pw))
        else:
            r_order, po = _arr(r_order, np.int32)
            self._check(lib().tnvan_set_width_set_ordered(self._h, instance, w.shape[0], pw, po))

    def set_made(self, instance: int, hidden: Sequence[int], d_params):
        h, ph = _arr(list(hidden) if len(hidden) else [0], np.int32)
        self._check(lib().tnvan_set_made(self._h, instance, len(hidden), ph, _ptr(d_params)))

    def n_params(self, instance: int):
        n, off = ctypes.c_int64(), ctypes.c_int64()
        self._check(lib().tnvan_n_params(self._h, instance, ctypes.byref(n), ctypes.byref(off)))
        return n.value, off.value

    def instance_info(self, instance: int):
        info = (ctypes.c_int32 * 13)()
        self._check(lib().tnvan_instance_info(self._h, instance, info))
        keys = ["n_spins", "n_edges", "D", "kind", "n_components", "max_component", "max_width", "n_ww",
                "arena", "arena_live", "tcg_slots", "fused_bwd", "tcg_streamed"]
        return dict(zip(keys, list(info)))

    def reserve(self, max_batch: int):
        self._check(lib().tnvan_reserve(self._h, max_batch))

    # --- hot path ---------------------------------------------------------
    def sample_and_contract(self, betas, batch: int, seed: int, step: int, precision: int, spins, logq,
                            logZR, stream=None):
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_sample_and_contract(self._h, pb, batch, seed, step, precision, _ptr(spins),
                                                    _ptr(logq), _ptr(logZR), _stream(stream)))

    def sample_contract_adjoint(self, betas, batch: int, seed: int, step: int, precision: int, spins, logq,
                                logZR, dbeta=None, dJ=None, stream=None):
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_sample_contract_adjoint(self._h, pb, batch, seed, step, precision, _ptr(spins),
                                                        _ptr(logq), _ptr(logZR), _ptr(dbeta), _ptr(dJ),
                                                        _stream(stream)))

    def train_step(self, betas, batch: int, seed: int, step: int, precision: int, spins, logq, logZR, dbeta, dJ,
                   grad, m, v, lr: float, beta1: float, beta2: float, eps: float, t: int, stream=None):
        """Sampling with the contraction adjoint, the REINFORCE gradient and
        Adam on the networks' own parameters, in one call."""
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_train_step(self._h, pb, batch, seed, step, precision, _ptr(spins), _ptr(logq),
                                           _ptr(logZR), _ptr(dbeta), _ptr(dJ), _ptr(grad), _ptr(m), _ptr(v),
                                           lr, beta1, beta2, eps, t, _stream(stream)))

    def log_prob(self, batch: int, spins, logq, precision: int = FP32, stream=None):
        self._check(lib().tnvan_log_prob(self._h, batch, _ptr(spins), precision, _ptr(logq), _stream(stream)))

    def contract(self, betas, batch: int, spins, precision: int, logZR, dlogZR_dbeta=None, stream=None):
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_contract(self._h, pb, batch, _ptr(spins), precision, _ptr(logZR),
                                         _ptr(dlogZR_dbeta), _stream(stream)))

    def observables(self, betas, batch: int, spins, logZR, logq, corr=None, stream=None) -> np.ndarray:
        """[n_inst, 3]: importance-weighted internal energy U, its mean under q,
        and the weights' effective sample size; with `corr` (device double
        [sum n_edges]) also the weighted beta * <s_i s_j> per edge."""
        b, pb = _arr(betas, np.float64)
        out = np.zeros(3 * len(b))
        self._check(lib().tnvan_observables(self._h, pb, batch, _ptr(spins), _ptr(logZR), _ptr(logq), _ptr(corr),
                                            out.ctypes.data_as(_dblp), _stream(stream)))
        return out.reshape(len(b), 3)

    def magnetisation(self, betas, batch: int, spins, logZR, logq, mag_mean=None, mag_var=None,
                      stream=None) -> np.ndarray:
        """[n_inst, 6]: importance-weighted <M>, <M^2>, the susceptibility per
        spin beta (<M^2> - <M>^2) / N, <M> and <M^2> under q, and the weights'
        effective sample size; with `mag_mean` / `mag_var` (device double
        [n_inst * batch]) also each sample's E[M | s] and Var(M | s)."""
        b, pb = _arr(betas, np.float64)
        out = np.zeros(6 * len(b))
        self._check(lib().tnvan_magnetisation(self._h, pb, batch, _ptr(spins), _ptr(logZR), _ptr(logq),
                                              _ptr(mag_mean), _ptr(mag_var), out.ctypes.data_as(_dblp),
                                              _stream(stream)))
        return out.reshape(len(b), 6)

    def free_energy(self, betas, batch: int, logZR, logq, stream=None) -> np.ndarray:
        b, pb = _arr(betas, np.float64)
        out = np.zeros(4 * len(b))
        _, po = _arr(out, np.float64)
        self._check(lib().tnvan_free_energy(self._h, pb, batch, _ptr(logZR), _ptr(logq),
                                            out.ctypes.data_as(_dblp), _stream(stream)))
        return out.reshape(len(b), 4)

    def reduce(self, betas, batch: int, logZR, logq, stats_out=None, stream=None):
        """Eq. 9 rows [8 per instance] into the context (and stats_out), async."""
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_reduce(self._h, pb, batch, _ptr(logZR), _ptr(logq), _ptr(stats_out),
                                       _stream(stream)))

    def step_stats(self, stats_out, stream=None):
        """The context's step statistics (last training step, reduce or merge) into stats_out."""
        self._check(lib().tnvan_step_stats(self._h, _ptr(stats_out), _stream(stream)))

    def merge_stats(self, betas, parts, stats_out=None, stream=None):
        """Statistics rows of disjoint parts [n_parts, n_inst * 8] merged into the context's."""
        b, pb = _arr(betas, np.float64)
        n_parts = parts.shape[0] if parts.dim() > 1 else parts.numel() // (8 * len(b))
        self._check(lib().tnvan_merge_stats(self._h, pb, n_parts, _ptr(parts), _ptr(stats_out), _stream(stream)))

    def backward_stats(self, betas, batch: int, spins, logZR, logq, precision: int, grad, stream=None):
        """Eq. 10 with the baseline and batch size of the context's step statistics."""
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_backward_stats(self._h, pb, batch, _ptr(spins), _ptr(logZR), _ptr(logq),
                                               precision, _ptr(grad), _stream(stream)))

    def backward(self, betas, batch: int, spins, logZR, logq, precision: int, grad, dlogZR_dbeta=None,
                 dlogZR_dJ=None, stream=None):
        b, pb = _arr(betas, np.float64)
        self._check(lib().tnvan_backward(self._h, pb, batch, _ptr(spins), _ptr(logZR), _ptr(logq), precision,
                                         _ptr(grad), _ptr(dlogZR_dbeta), _ptr(dlogZR_dJ), _stream(stream)))

    def set_step_counter(self, counter):
        self._check(lib().tnvan_set_step_counter(self._h, None if counter is None else _ptr(counter)))

    def autotune(self, betas, batch: int, precision: int, stream=None):
        """Time candidate launch shapes on a synthetic batch and keep the fastest;
        returns the chosen (sampler tile, strip tile, backward CTAs, strip adjoint tile,
        tensor-core sampler plan (grouped form: 4, 6, 8 steps per group; per-step
        form: 12, 16, 32 steps per chunk), overlapped schedule 2 on / 1 off, backward
        form of networks without the fused kernel 1 tensor-core chain / 2 FP32 SIMT)."""
        b, pb = _arr(betas, np.float64)
        out = (ctypes.c_int32 * 7)()
        self._check(lib().tnvan_autotune(self._h, pb, batch, precision, _stream(stream), out))
        return tuple(out[:7])

    def set_tuning(self, choices):
        """Reuse launch shapes (the 7-tuple autotune returns; 0 = default; a
        6-tuple leaves the backward form at its default)."""
        c = list(choices)
        if len(c) == 6:
            c.append(0)
        c, pc = _arr(c, np.int32)
        if c.shape[0] != 7:
            raise ValueError("expected 6 or 7 tuning values")
        self._check(lib().tnvan_set_tuning(self._h, pc))

    def profile(self, enable: bool):
        self._check(lib().tnvan_profile(self._h, int(enable)))

    def profile_trace(self):
        """[(kernel index, start ms, end ms)] of every recorded launch, relative to
        the start of the profiled region (call before profile_read)."""
        n = ctypes.c_int64()
        self._check(lib().tnvan_profile_trace(self._h, 0, None, None, None, ctypes.byref(n)))
        m = n.value
        kk = np.zeros(m, np.int32)
        a = np.zeros(m, np.float32)
        b = np.zeros(m, np.float32)
        self._check(lib().tnvan_profile_trace(self._h, m, kk.ctypes.data, a.ctypes.data, b.ctypes.data,
                                              ctypes.byref(n)))
        return list(zip(kk.tolist(), a.tolist(), b.tolist()))

    def profile_read(self):
        """{kernel name: (total ms, launches)} of the recorded launches."""
        out = {}
        k = 0
        buf = ctypes.create_string_buffer(64)
        while True:
            ms, n = ctypes.c_double(), ctypes.c_int64()
            rc = lib().tnvan_profile_read(self._h, k, buf, 64, ctypes.byref(ms), ctypes.byref(n))
            if rc == E_ARG:
                break
            self._check(rc)
            out[buf.value.decode()] = (ms.value, n.value)
            k += 1
        return out

    def adam(self, params, grad, m, v, lr: float, beta1: float, beta2: float, eps: float, t: int, stream=None):
        self._check(lib().tnvan_adam(self._h, params.numel(), _ptr(params), _ptr(grad), _ptr(m), _ptr(v),
                                     lr, beta1, beta2, eps, t, _stream(stream)))
