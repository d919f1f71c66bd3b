"""The allocation-free free-energy entry point, for callers that may not
allocate device memory (an external memory manager, a plugin with a fixed
device footprint, a path where cudaMalloc's synchronisation is not allowed).

It is called through the C-ABI and must agree with the context-based
tnvan_free_energy on two calls in a row (the second call reuses the shared
scratch array left by the first), and with an FP64 NumPy evaluation of the
same estimators when some l_b are non-finite (they are left out), when an
instance has no finite l_b, at the 128-instance limit with many chunks per
instance, and for a batch of one.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(betas, batch, logZR, logq):
    L = tv.lib()
    betas = np.ascontiguousarray(betas, np.float64)
    out = torch.full((5 * len(betas),), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.tnvan_free_energy_noalloc(len(betas), batch, betas.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     logZR.data_ptr(), logq.data_ptr(), out.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert rc == tv.OK, L.tnvan_noalloc_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(len(betas), 5)


def test_noalloc_free_energy_matches_context_version_twice():
    from paper_2504_12037_gb300.model import TNVAN

    w = wl.workload(2)
    model = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, seed=5)
    rng = np.random.default_rng(17)
    for call, B in enumerate((3000, 777)):
        lz = torch.as_tensor(rng.normal(-250 + 10 * call, 4, size=model.n * B)).cuda()
        lq = torch.as_tensor(rng.normal(-40, 3, size=model.n * B).astype(np.float32)).cuda()
        ref = model.ctx.free_energy(model.betas, B, lz, lq)
        got = _noalloc(model.betas, B, lz, lq)
        for k in range(model.n):
            N = w.graphs[k].n
            assert abs(got[k, 0] - ref[k, 0]) / N < 1e-9
            assert abs(got[k, 1] - ref[k, 1]) / N < 1e-9
            assert abs(got[k, 3] - ref[k, 3]) / N < 1e-9
            assert abs(got[k, 2] - ref[k, 2]) <= 1e-9 * abs(ref[k, 2])
            assert got[k, 4] == 0


def test_noalloc_rejects_too_many_instances():
    L = tv.lib()
    betas = np.ones(129)
    buf = torch.zeros(129 * 4, dtype=torch.float64, device="cuda")
    rc = L.tnvan_free_energy_noalloc(129, 4, betas.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None)
    assert rc == tv.E_ARG
    assert b"128" in L.tnvan_noalloc_last_error()


def _np_stats(lz, lq, beta):
    """F_q, F_IS, stderr, logZ_IS and the non-finite count of one instance, FP64."""
    l = lz - lq.astype(np.float64)
    ok = np.isfinite(l)
    f = l[ok]
    n = f.size
    if n == 0:
        return np.array([np.nan] * 4 + [float(l.size)])
    m = f.max()
    lzis = m + np.log(np.exp(f - m).sum()) - np.log(n)
    se = f.std(ddof=1) / (beta * np.sqrt(n)) if n > 1 else 0.0
    return np.array([-f.mean() / beta, -lzis / beta, se, lzis, float(l.size - n)])


def _check(got, want, N=64):
    for k in range(want.shape[0]):
        assert got[k, 4] == want[k, 4]
        if np.isnan(want[k, 0]):
            assert np.all(np.isnan(got[k, :4]))
            continue
        assert abs(got[k, 0] - want[k, 0]) / N < 1e-9
        assert abs(got[k, 1] - want[k, 1]) / N < 1e-9
        assert abs(got[k, 3] - want[k, 3]) / N < 1e-9
        assert abs(got[k, 2] - want[k, 2]) <= 1e-9 * abs(want[k, 2]) + 1e-300


def test_noalloc_non_finite_samples_left_out():
    # one row of NaN, -inf at the first sample of an instance, +inf elsewhere,
    # and an instance whose every l_b is non-finite
    rng = np.random.default_rng(3)
    n_inst, B = 4, 2500
    betas = np.array([0.5, 1.0, 1.5, 2.0])
    lz = rng.normal(-120, 3, size=(n_inst, B))
    lq = rng.normal(-30, 2, size=(n_inst, B)).astype(np.float32)
    lz[0, 0] = -np.inf
    lz[1, 17] = np.nan
    lq[1, 2499] = np.inf
    lz[2, :] = np.nan
    lz[3, 1024] = np.inf
    want = np.stack([_np_stats(lz[k], lq[k], betas[k]) for k in range(n_inst)])
    got = _noalloc(betas, B, torch.as_tensor(lz.ravel()).cuda(), torch.as_tensor(lq.ravel()).cuda())
    assert list(got[:, 4]) == [1, 2, B, 1]
    _check(got, want)


def test_noalloc_many_instances_many_chunks_and_batch_one():
    # 128 instances (the limit) with 17,000 samples each: more chunks per
    # instance than the shared tuple array holds, so the chunk count is capped
    rng = np.random.default_rng(4)
    n_inst, B = 128, 17000
    betas = rng.uniform(0.2, 2.0, n_inst)
    lz = rng.normal(-200, 5, size=(n_inst, B))
    lq = rng.normal(-40, 3, size=(n_inst, B)).astype(np.float32)
    want = np.stack([_np_stats(lz[k], lq[k], betas[k]) for k in range(n_inst)])
    got = _noalloc(betas, B, torch.as_tensor(lz.ravel()).cuda(), torch.as_tensor(lq.ravel()).cuda())
    _check(got, want)
    # a batch of one sample per instance: stderr 0, F_IS = F_q
    lz1, lq1 = lz[:, :1].copy(), lq[:, :1].copy()
    got = _noalloc(betas, 1, torch.as_tensor(lz1.ravel()).cuda(), torch.as_tensor(lq1.ravel()).cuda())
    want = np.stack([_np_stats(lz1[k], lq1[k], betas[k]) for k in range(n_inst)])
    _check(got, want)
    assert np.all(got[:, 2] == 0.0)
