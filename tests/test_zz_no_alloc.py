"""xlmimo_channel_gram_noalloc: the Gram entry point for callers that cannot
allocate device memory while they run (a host that has reserved the GPU's
memory for its own pool, or a latency-critical loop that cannot accept
cudaMalloc / cudaFree).  It must give what xlmimo_channel_gram gives, call
after call, using only its fixed device scratch.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2503_18118_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LAM100 = inputs.wavelength(100e9)


def normwise(G, Gref):
    d = np.sqrt(np.abs(np.einsum("...ii->...i", Gref)))
    return float(np.max(np.abs(G - Gref) / (d[..., :, None] * d[..., None, :])))


def test_noalloc_source_allocates_nothing():
    """The entry point's file calls no allocator (static check, no GPU)."""
    text = open(os.path.join(ROOT, "paper_2503_18118_gb300", "csrc", "gram_noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", text)
    for word in ("cudaMalloc", "cudaFree", "malloc(", "new "):
        assert word not in code, word
    src = open(os.path.join(ROOT, "paper_2503_18118_gb300", "csrc", "gram_simt.cu")).read()
    body = src[src.index("int launch_gram_into_scratch"):]
    assert "cudaMalloc" not in body and "cudaFree" not in body


@pytest.mark.gpu
def test_noalloc_matches_channel_gram_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18118_gb300 import xlmimo as xl
    N, K = 70001, 8  # two trials over 70001 elements: the element range is split
    arr = xl.array(N, LAM100, None, 1.0, xl.FSPL_USW)
    for prec in (xl.F64, xl.F32):
        for call, seed in enumerate((41, 42)):  # two calls in a row, different users
            users = torch.from_numpy(inputs.users_polar(seed, 2, K, (3.0, 30.0))).cuda()
            ref = xl.xlmimo_channel_gram(arr, users, prec)
            out = torch.full_like(ref, complex(float("nan"), float("nan")))
            xl.xlmimo_channel_gram_noalloc(arr, users, prec, out)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.isfinite(a).all()
            if prec == xl.F64:
                u = users.cpu().numpy()
                rmax = float(np.hypot(u[..., 0], np.abs(u[..., 1]) + N * LAM100 / 4).max())
                tol = max(1e-12, 8 * np.finfo(float).eps * (1 + 2 * math.pi * rmax / LAM100) / math.sqrt(N))
            else:
                tol = 1e-5
            assert normwise(a, b) <= tol, (prec, call)


@pytest.mark.gpu
def test_noalloc_rejects_oversized_split():
    """A batch whose element split needs more than the static scratch is
    refused on the host.  Real device buffers of the call's shapes are passed,
    so that even a call that were accepted would touch only valid memory."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18118_gb300 import xlmimo as xl
    N, K, B = 1 << 22, 64, 1
    # the split the library chooses (element tiles of 128 for FP32; at least
    # two tiles per chunk; at most 4096 chunks) and the scratch it then needs
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = N // 128
    S = min(max(min(-(-4 * sms // B), tiles // 2), 1), 4096)
    chunk = -(-tiles // S) * 128
    S = -(-N // chunk)
    need = B * S * K * K * 16
    if need <= xl.NOALLOC_SCRATCH_MIB << 20:
        pytest.skip(f"{sms} SMs: this split fits the scratch")
    L = xl.lib()
    arr = xl.array(N, LAM100, None, 1.0, xl.FSPL_USW)
    users = torch.from_numpy(inputs.users_polar(43, B, K, (3.0, 30.0))).cuda()
    gram = torch.zeros((B, K, K), dtype=torch.complex128, device="cuda")
    rc = L.xlmimo_channel_gram_noalloc(ctypes.byref(arr), ctypes.c_void_p(users.data_ptr()), K, B, xl.F32,
                                       ctypes.c_void_p(gram.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == 1
    assert b"scratch" in L.xlmimo_last_error()
