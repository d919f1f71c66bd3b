"""Without a GPU the product path fails loudly: no CPU fallback (CPU only;
skipped where a GPU is present)."""
import os

import pytest
import torch

from paper_2504_12037_gb300 import tnvan as tv
from paper_2504_12037_gb300 import workloads as wl

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(tv.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()


def test_model_refuses_to_run_without_a_gpu():
    from paper_2504_12037_gb300.model import TNVAN

    w = wl.workload(1)
    with pytest.raises(RuntimeError):
        TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas)


def test_library_context_reports_a_cuda_error():
    with pytest.raises(tv.TnvanError) as e:
        tv.Context(0)
    assert e.value.code == tv.E_CUDA


def test_host_only_finder_still_runs():
    g = wl.random_regular(60, 3, 5)
    W, order, width, _ = tv.find_width_set(g.n, g.ei, g.ej, 2)
    assert width <= 2 and len(W) + len(order) == g.n
