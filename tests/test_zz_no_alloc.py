"""The allocation-free entry point (tsk_approx_noalloc), through the C ABI.

It exists for callers that cannot allocate device memory where they need an
approximation (inside another framework's memory pool, on latency-critical
paths, under a fixed memory budget).  It must give what the allocating entry
point (tsk_approx_batch) gives, within the tolerances the other tests use,
and do so again on a second call in a row: the static scratch array keeps
the previous call's contents, so anything that accumulates must be cleared.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2209_14637_gb300 as mod
    from paper_2209_14637_gb300 import build
    build.build()
    mod.load_library()
    return mod


def _noalloc(tsk, A, S, r, prec):
    lib = tsk.load_library()
    d = tsk.MatDesc(A.data_ptr(), S.data_ptr(), A.shape[0], A.shape[1], A.stride(0),
                    S.shape[0], r)
    err = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    nrm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    st = lib.tsk_approx_noalloc(C.byref(d), prec, C.c_void_p(err.data_ptr()),
                                C.c_void_p(nrm.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, float(err.item()), float(nrm.item())


@pytest.mark.parametrize("dtype,m,n,k,r,tol", [
    (torch.float64, 128, 96, 10, 5, 1e-10),
    (torch.float32, 1024, 768, 20, 10, 1e-3),
    (torch.bfloat16, 520, 392, 16, 8, 1e-3),
])
def test_noalloc_matches_allocating_entry(tsk, dtype, m, n, k, r, tol):
    g = torch.Generator(device="cuda").manual_seed(m + n)
    L = 2 * k
    U = torch.linalg.qr(torch.randn(m, L, generator=g, device="cuda",
                                    dtype=torch.float64))[0]
    sv = torch.arange(1, L + 1, device="cuda", dtype=torch.float64) ** -1.2
    A = ((U * sv) @ torch.randn(L, n, generator=g, device="cuda", dtype=torch.float64)
         + 1e-3 * torch.randn(m, n, generator=g, device="cuda", dtype=torch.float64))
    A = A.to(dtype).contiguous()
    sdt = torch.float64 if dtype == torch.float64 else torch.float32
    S = torch.linalg.qr(U[:, :k] + 0.1 * torch.randn(m, k, generator=g, device="cuda",
                                                      dtype=torch.float64))[0].T
    S = S.to(sdt).contiguous()
    prec = {torch.float64: tsk.FP64, torch.float32: tsk.FP32, torch.bfloat16: tsk.BF16}[dtype]
    h = tsk.Handle()
    ref = h.approx_batch([A], [S], r)
    torch.cuda.synchronize()
    e_ref, n_ref = float(ref["err"][0]), float(ref["normA2"][0])
    h.close()
    results = [_noalloc(tsk, A, S, r, prec) for _ in range(2)]  # two calls in a row
    for st, e, nrm in results:
        assert st == 0, tsk.load_library().tsk_last_error(None)
        assert abs(e - e_ref) <= tol * e_ref, (e, e_ref)
        assert abs(nrm - n_ref) <= max(tol, 1e-6) * n_ref, (nrm, n_ref)
    assert abs(results[0][1] - results[1][1]) <= 1e-12 * results[0][1]


def test_noalloc_rejects_sizes_beyond_its_array(tsk):
    lib = tsk.load_library()
    # (m + n) * k_pad * 4 bytes = 70000 * 64 * 4 > 8 MiB; the call is rejected
    # from the sizes alone, before anything reads the (tiny) buffer
    buf = torch.empty(64, device="cuda")
    d = tsk.MatDesc(buf.data_ptr(), buf.data_ptr(), 35000, 35000, 35000, 64, 8)
    err = torch.empty(1, dtype=torch.float64, device="cuda")
    st = lib.tsk_approx_noalloc(C.byref(d), tsk.FP32, C.c_void_p(err.data_ptr()), None, None)
    assert st == 1  # TSK_EINVAL, rejected before any device work
    assert b"static array" in lib.tsk_last_error(None)
