"""The allocation-free free-energy entry point, for callers that may not
allocate device memory (an external memory manager, a plugin with a fixed
device footprint, a path where cudaMalloc's synchronisation is not allowed).

It is called through the C-ABI and must agree with the context-based
tnvan_free_energy on two calls in a row (the second call reuses the shared
scratch array left by the first).  Collected last on purpose."""
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
