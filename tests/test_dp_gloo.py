"""The data-parallel exchange (dp.py) with world_size-2 gloo ranks on the CPU.

Each rank holds a disjoint share of one batch and its Eq. 9 statistics rows
in the device reduction's layout (F_q, F_IS, stderr, logZ_IS, mean l,
#non-finite, var l, n).  After the all-gather and the rank-order merge, every
rank must hold the oracle's statistics of the union batch; the REINFORCE
gradients each rank forms with the merged baseline and batch size must sum
(all-reduce) to the oracle's gradient of the union batch."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

BETAS = [0.4, 1.3]
D, HIDDEN = 5, [7, 6]
SIZES = (500, 800)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_data(rank, k):
    """Rank `rank`'s samples of instance k: spins [n, D], log Z_R, log q."""
    from oracle import made

    rng = np.random.default_rng(1000 * k + rank)
    n = SIZES[rank]
    s = torch.as_tensor(rng.choice([-1.0, 1.0], size=(n, D)))
    th = torch.as_tensor(made.init_params(D, HIDDEN, 11 + k))
    lq = made.log_q(th, D, HIDDEN, s)
    lz = torch.as_tensor(rng.normal(-60 + 20 * k, 2 + rank, size=n))
    return s, lz, lq, th


def _rows(lz, lq, beta):
    """Statistics row of one instance's samples in the reduction's layout (oracle)."""
    from oracle import estimators as est

    r = est.free_energies(lz, lq, beta)
    l = (lz - lq).numpy()
    return np.array([r["F_q"], r["F_IS"], r["stderr"], r["logZ_IS"], l.mean(), 0.0, l.var(ddof=1), l.size])


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import estimators as est
        from paper_2504_12037_gb300 import dp

        local = torch.as_tensor(np.stack([_rows(*_rank_data(rank, k)[1:3], BETAS[k]) for k in range(2)]))
        parts = dp.gather_stats(local)
        merged = dp.merge_stats(parts.numpy(), BETAS)
        grads = []
        for k in range(2):
            s, lz, lq, th = _rank_data(rank, k)
            # Eq. 10 on this rank's samples with the merged baseline and batch size
            w = -((lz - lq) - merged[k, dp.MEAN]) / (BETAS[k] * merged[k, dp.N])
            grads.append(est.surrogate_grad(th.numpy(), D, HIDDEN, s, w))
        g = torch.cat(grads)
        dp.sum_gradient(g)
        q.put((rank, parts.numpy(), merged, g.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_and_gradient_match_oracle_on_union():
    from oracle import estimators as est
    from paper_2504_12037_gb300 import dp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    g_ref = []
    for k, b in enumerate(BETAS):
        data = [_rank_data(r, k) for r in range(2)]
        s = torch.cat([d[0] for d in data])
        lz = torch.cat([d[1] for d in data])
        lq = torch.cat([d[2] for d in data])
        ref = _rows(lz, lq, b)
        for rank in range(2):
            m = res[rank][2][k]
            for j in (dp.F_Q, dp.F_IS, dp.LOGZ_IS, dp.MEAN):
                assert abs(m[j] - ref[j]) <= 1e-12 * abs(ref[j]), (k, j)
            for j in (dp.STDERR, dp.VAR):
                assert abs(m[j] - ref[j]) <= 1e-10 * ref[j], (k, j)
            assert m[dp.N] == sum(SIZES) and m[dp.BAD] == 0
        g_ref.append(est.surrogate_grad(data[0][3].numpy(), D, HIDDEN, s, est.reinforce_weights(lz, lq, b)))
    g_ref = torch.cat(g_ref).numpy()
    for rank in range(2):
        assert np.abs(res[rank][3] - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
        # the gathered parts are each rank's own rows, in rank order
        for r in range(2):
            for k in range(2):
                assert np.array_equal(res[rank][1][r, k], _rows(*_rank_data(r, k)[1:3], BETAS[k]))
    assert np.array_equal(res[0][2], res[1][2])  # identical on every rank
    assert np.array_equal(res[0][3], res[1][3])


def test_merge_of_one_part_is_the_part_and_order_free_counts():
    from paper_2504_12037_gb300 import dp

    rng = np.random.default_rng(2)
    rows = rng.normal(size=(1, 3, 8))
    rows[..., dp.N] = [10, 1, 7]
    assert np.array_equal(dp.merge_stats(rows, [1.0, 2.0, 3.0]), rows[0])
    # a part with no finite samples only adds its non-finite count
    a = np.array([[[-1.0, -1.2, 0.1, 1.2, 1.0, 0.0, 0.5, 40.0]]])
    e = np.array([[[np.nan] * 4 + [np.nan, 3.0, np.nan, 0.0]]])
    m = dp.merge_stats(np.concatenate([a, e]), [1.0])
    assert np.allclose(m[0, [0, 1, 3, 4, 6, 7]], a[0, 0, [0, 1, 3, 4, 6, 7]], rtol=1e-14, atol=0)
    assert m[0, dp.BAD] == 3.0
