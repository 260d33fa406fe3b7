"""Multi-process (gloo, world size 2, CPU) combination of per-chain estimator
rows and timings: pooling rows gathered from two ranks equals pooling all rows
in one process, bitwise; the timing is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest


def _stat_rows(series_list):
    """Per-chain rows built by the accumulation rule of the estimator:
    running sums and batch sums with doubling batch length (32..64 batches)."""
    from paper_1403_0711_gb300 import coulps
    rows = []
    for e in series_list:
        st = np.zeros(coulps.STAT_STRIDE)
        st[5] = 1.0
        for v in e:
            st[0] += 1; st[1] += v; st[2] += v * v; st[3] += v; st[4] += 1
            if st[4] >= st[5]:
                nb = int(st[6])
                st[8 + nb] = st[3]; st[3] = 0; st[4] = 0
                nb += 1
                if nb == 64:
                    for i in range(32):
                        st[8 + i] = st[8 + 2 * i] + st[8 + 2 * i + 1]
                    st[8 + 32:8 + 64] = 0
                    nb = 32
                    st[5] *= 2
                st[6] = nb
        rows.append(st)
    return np.array(rows)


def _series(n_chains, n, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n) * 2 + 0.5 for _ in range(n_chains)]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1403_0711_gb300 import dist as cdist
    rows = _stat_rows(_series(3, 1000, seed=10 + rank))
    est = cdist.pooled_estimate(rows)
    t = cdist.max_over_ranks(1.5 + rank)
    q.put((rank, est, t))
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_pool_over_two_gloo_ranks():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    coulps.load()
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
    single = coulps.pool_stats(np.concatenate([_stat_rows(_series(3, 1000, seed=10)),
                                               _stat_rows(_series(3, 1000, seed=11))]))
    for rank, est, t in res:
        assert est == single
        assert t == 2.5
    # the pooled mean is the plain mean of all samples
    allv = np.concatenate(_series(3, 1000, 10) + _series(3, 1000, 11))
    assert abs(single["mean"] - allv.mean()) < 1e-12
    assert single["n"] == 6000


def test_pool_rejects_mixed_batch_lengths():
    from paper_1403_0711_gb300 import _build, coulps
    _build.build()
    coulps.load()
    a = _stat_rows(_series(1, 1000, 1))
    b = _stat_rows(_series(1, 100, 2))
    with pytest.raises(coulps.CoulpsError):
        coulps.pool_stats(np.concatenate([a, b]))
