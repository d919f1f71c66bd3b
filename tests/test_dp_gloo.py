"""Multi-rank exchange (dp.py) with world_size-2 gloo ranks on the CPU: the
merged statistics equal the oracle estimators over the union of the ranks'
samples, and the gradient average is exact."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import estimators as est
        from paper_2504_12037_gb300 import dp

        betas = [0.4, 1.3]
        rng = np.random.default_rng(100 + rank)
        n_local = 500 + 300 * rank
        fe = np.zeros((2, 4))
        for k, b in enumerate(betas):
            l = rng.normal(-200 + 50 * k, 3 + rank, size=n_local)
            r = est.free_energies(l, np.zeros(n_local), b)  # rank-local statistics (the device reduction's output)
            fe[k] = [r["F_q"], r["F_IS"], r["stderr"], r["logZ_IS"]]
        merged = dp.allreduce_free_energy(fe, n_local, betas)
        g = torch.full((7,), float(rank + 1))
        dp.allreduce_gradient(g)
        q.put((rank, merged, g.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_matches_oracle_on_union():
    from oracle import estimators as est

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    # rebuild the union of both ranks' samples
    betas = [0.4, 1.3]
    for k, b in enumerate(betas):
        ls = []
        for rank in range(2):
            rng = np.random.default_rng(100 + rank)
            n_local = 500 + 300 * rank
            for kk in range(k + 1):
                l = rng.normal(-200 + 50 * kk, 3 + rank, size=n_local)
            ls.append(l)
        allv = np.concatenate(ls)
        ref = est.free_energies(allv, np.zeros_like(allv), b)
        for rank in range(2):
            m = res[rank][1][k]
            assert abs(m[0] - ref["F_q"]) < 1e-10 * abs(ref["F_q"])
            assert abs(m[1] - ref["F_IS"]) < 1e-10 * abs(ref["F_IS"])
            assert abs(m[2] - ref["stderr"]) < 1e-8 * ref["stderr"]
            assert abs(m[3] - ref["logZ_IS"]) < 1e-10 * abs(ref["logZ_IS"])
    for rank in range(2):
        assert np.allclose(res[rank][2], 1.5)
    assert np.array_equal(res[0][1], res[1][1])  # identical on every rank
