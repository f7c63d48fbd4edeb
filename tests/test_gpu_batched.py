"""Ragged batches (instances with their own N, K, receiver and noise) through
the plan / run C entry points, against the FP64 oracle per instance; CUDA
graph capture and replay; the autotuned plan."""
import math

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM = inputs.wavelength(100e9)


@pytest.fixture(scope="module")
def xl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18118_gb300 import xlmimo
    xlmimo.lib()
    return xlmimo


def normwise(G, Gref):
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Gref)))
    return float(np.max(np.abs(G - Gref) / (d[..., :, None] * d[..., None, :])))


def make_batch(seed, count, n_range=(256, 40000), k_range=(1, 64)):
    g = np.random.Generator(np.random.Philox(key=seed))
    n = np.rint(np.exp(g.uniform(np.log(n_range[0]), np.log(n_range[1]), count))).astype(np.int64)
    k = g.integers(k_range[0], k_range[1] + 1, count)
    scheme = g.integers(0, 2, count)
    noise = g.uniform(0.5, 2.0, count)
    users = inputs.users_polar(seed + 1, 1, int(k.sum()), (3.0, 30.0))[0]
    snr = 10 ** (g.uniform(0.0, 30.0, int(k.sum())) / 10)
    return n, k, scheme, noise, users, snr


def run_plan(xl, plan, users, snr):
    U, n = plan.users_total, plan.count
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = dict(gram=torch.empty(plan.gram_total, dtype=torch.complex128, device="cuda"),
               sinr=torch.empty(U, dtype=torch.float64, device="cuda"),
               status=torch.empty(n, dtype=torch.int32, device="cuda"),
               rate=torch.empty(n, dtype=torch.float64, device="cuda"))
    plan.run(dev(users), dev(snr), xl.POWER_RXSNR, **out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("prec,gtol", [(3, 1e-4), (4, 5e-4), (2, 1e-2)])
def test_batch_matches_oracle(xl, orc, prec, gtol):
    n, k, scheme, noise, users, snr = make_batch(11, 60)
    arr = xl.array(1, LAM)
    plan = xl.BatchPlan(arr, n, k, scheme, noise, prec=prec)
    info = plan.info()
    assert info["items"] >= len(n) and info["small"] + info["large"] == len(n)
    out = run_plan(xl, plan, users, snr)
    for i in range(len(n)):
        K, uo, go = int(k[i]), int(plan.user_off[i]), int(plan.gram_off[i])
        u = users[uo:uo + K][None]
        G = out["gram"][go:go + K * K].reshape(1, K, K)
        R = orc.gram(orc.FSPL, int(n[i]), LAM, LAM / 2, 1.0, u)
        assert normwise(G, R) <= gtol, i
        # receiver and rate on the same (GPU) Gram: FP64 solves on both sides,
        # agreeing to the FP64 rounding amplified by the Gram's conditioning
        s_ref, st_ref, _ = orc.beamform(G, snr[uo:uo + K][None], noise[i:i + 1], int(scheme[i]), orc.POWER_RXSNR)
        s = out["sinr"][uo:uo + K]
        tol = max(1e-9, 1e-14 * np.linalg.cond(G[0]))
        if st_ref[0] == 0:
            assert np.max(np.abs(s - s_ref[0]) / np.abs(s_ref[0])) <= tol, i
            assert abs(out["rate"][i] - np.log2(1 + s_ref[0]).sum()) <= tol * abs(out["rate"][i]), i


def test_batch_split_instances(xl, orc):
    """Instances longer than the element chunk are split into work items whose
    partial Gram matrices are summed in chunk order."""
    n = np.array([200000, 70001, 5, 131072])
    k = np.array([3, 40, 2, 64])
    users = inputs.users_polar(5, 1, int(k.sum()), (3.0, 30.0))[0]
    arr = xl.array(1, LAM)
    plan = xl.BatchPlan(arr, n, k, np.zeros(4), np.ones(4))
    assert plan.info()["items"] > 4
    out = run_plan(xl, plan, users, np.full(int(k.sum()), 10.0))
    for i in range(4):
        K, uo, go = int(k[i]), int(plan.user_off[i]), int(plan.gram_off[i])
        G = out["gram"][go:go + K * K].reshape(1, K, K)
        R = orc.gram(orc.FSPL, int(n[i]), LAM, LAM / 2, 1.0, users[uo:uo + K][None])
        assert normwise(G, R) <= 1e-4, i


def test_batch_graph_capture_and_autotune(xl):
    """The run enqueues kernels only, so it captures into a CUDA graph; replays
    reproduce a direct run exactly.  The autotuned plan picks one of its
    candidates."""
    n, k, scheme, noise, users, snr = make_batch(12, 300, (1024, 131072), (2, 64))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    U = dev(users)
    arr = xl.array(1, LAM)
    plan = xl.BatchPlan(arr, n, k, scheme, noise, tune_users=U)
    info = plan.info()
    assert info["tuned"] == 1 and info["candidates"] == 6
    assert info["chunk"] in (4096, 8192, 16384) and info["ctas_per_sm"] in (1, 2)
    P = dev(snr)
    out = dict(gram=torch.empty(plan.gram_total, dtype=torch.complex128, device="cuda"),
               sinr=torch.empty(plan.users_total, dtype=torch.float64, device="cuda"),
               status=torch.empty(plan.count, dtype=torch.int32, device="cuda"),
               rate=torch.empty(plan.count, dtype=torch.float64, device="cuda"))
    plan.run(U, P, xl.POWER_RXSNR, **out)
    torch.cuda.synchronize()
    ref = {kk: v.clone() for kk, v in out.items()}
    for v in out.values():
        v.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run(U, P, xl.POWER_RXSNR, **out, stream=s)
    for _ in range(2):
        for v in out.values():
            v.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for kk in ref:
            assert torch.equal(out[kk], ref[kk]), kk
