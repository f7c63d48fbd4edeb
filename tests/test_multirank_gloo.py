"""The multi-rank host logic (paper_2503_18118_gb300/mc.py) on CPU processes
with the gloo backend, world size 2: distinct trial blocks per rank, the
max-over-ranks time, the whole-job throughput, and the merge of per-rank
{mean, M2, count} statistics against the statistics of all trials."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2503_18118_gb300 import inputs, mc

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _stats(x):
    x = np.asarray(x, np.float64)
    m = x.mean()
    return np.array([m, float(((x - m) ** 2).sum()), float(x.size)])


def _rank_main(rank, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        users = inputs.users_polar(mc.rank_seed(3, rank), 64, 4, (3.0, 30.0))
        # per-trial "rates": any per-trial quantity, different sizes per rank
        rates = np.hypot(users[:, :, 0], users[:, :, 1]).sum(axis=1)[: 40 + 24 * rank]
        merged = mc.allgather_stats(_stats(rates), dist)
        t_ms = mc.max_over_ranks(10.0 + 5.0 * rank, dist)
        q.put((rank, users[0].tolist(), rates.tolist(), merged.tolist(), t_ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(WORLD):
        r, u0, rates, merged, t = q.get()
        res[r] = (np.array(u0), np.array(rates), np.array(merged), t)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # distinct trial blocks; rank 0's is the single-GPU run's
    assert not np.allclose(res[0][0], res[1][0])
    assert np.array_equal(res[0][0], inputs.users_polar(3, 64, 4, (3.0, 30.0))[0])
    # the slowest rank's time everywhere; throughput over it
    assert res[0][3] == res[1][3] == 15.0
    assert mc.throughput(WORLD, 100, 3, 15.0) == pytest.approx(2 * 100 * 3 / 0.015)
    # merged statistics = statistics of all trials, on every rank
    want = _stats(np.concatenate([res[0][1], res[1][1]]))
    for r in range(WORLD):
        assert np.allclose(res[r][2], want, rtol=1e-12, atol=1e-9)



def test_merge_stats_edge_cases():
    x = np.random.Generator(np.random.Philox(key=9)).normal(size=101)
    parts = [x[:0], x[:1], x[1:50], x[50:]]
    got = mc.merge_stats([_stats(p) if p.size else np.zeros(3) for p in parts])
    assert np.allclose(got, _stats(x), rtol=1e-12, atol=1e-12)
    assert np.array_equal(mc.merge_stats([]), np.zeros(3))
