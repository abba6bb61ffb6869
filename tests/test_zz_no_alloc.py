"""The allocation-free entry point (tsk_approx_noalloc), through the C ABI.

It exists for callers that cannot allocate device memory where they need an
approximation: code that runs inside another framework's memory pool,
latency-critical paths where cudaMalloc (which may synchronise the device)
is not allowed, and deployments with a fixed memory budget.  It must give
what the allocating entry point (tsk_approx_batch) gives, within the
tolerances the other tests use, and do so again on later calls: the static
scratch array keeps the previous call's contents, so anything that
accumulates must be cleared, including after a larger call or one in
another precision.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle

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
    sts = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = lib.tsk_approx_noalloc(C.byref(d), prec, C.c_void_p(err.data_ptr()),
                                C.c_void_p(nrm.data_ptr()), C.c_void_p(sts.data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, float(err.item()), float(nrm.item()), int(sts.item())


def _case(m, n, k, dtype, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    L = 2 * k
    U = torch.linalg.qr(torch.randn(m, L, generator=g, dtype=torch.float64))[0]
    sv = torch.arange(1, L + 1, dtype=torch.float64) ** -1.2
    A = (U * sv) @ torch.randn(L, n, generator=g, dtype=torch.float64) \
        + 1e-3 * torch.randn(m, n, generator=g, dtype=torch.float64)
    S = torch.linalg.qr(U[:, :k] + 0.1 * torch.randn(m, k, generator=g,
                                                      dtype=torch.float64))[0].T
    sdt = torch.float64 if dtype == torch.float64 else torch.float32
    return A.to(dtype).contiguous().cuda(), S.to(sdt).contiguous().cuda()


PREC = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}


def _reference(tsk, A, S, r):
    h = tsk.Handle()
    ref = h.approx_batch([A], [S], r)
    torch.cuda.synchronize()
    out = float(ref["err"][0]), float(ref["normA2"][0])
    h.close()
    return out


@pytest.mark.parametrize("dtype,m,n,k,r,tol", [
    (torch.float64, 128, 96, 10, 5, 1e-10),
    (torch.float32, 1024, 768, 20, 10, 1e-3),
    (torch.bfloat16, 520, 392, 16, 8, 1e-3),
])
def test_noalloc_matches_allocating_entry(tsk, dtype, m, n, k, r, tol):
    A, S = _case(m, n, k, dtype, m + n)
    e_ref, n_ref = _reference(tsk, A, S, r)
    results = [_noalloc(tsk, A, S, r, PREC[dtype]) for _ in range(2)]  # two calls in a row
    for st, e, nrm, sts in results:
        assert st == 0, tsk.load_library().tsk_last_error(None)
        assert sts == 0
        assert abs(e - e_ref) <= tol * e_ref, (e, e_ref)
        assert abs(nrm - n_ref) <= max(tol, 1e-6) * n_ref, (nrm, n_ref)
    assert abs(results[0][1] - results[1][1]) <= 1e-12 * results[0][1]


def test_noalloc_after_a_larger_call_and_another_precision(tsk):
    """A large FP32 call leaves its panels, descriptors and sums in the
    array; a following small FP64 call (another layout and element size)
    must not read any of it, nor a following BF16 call."""
    big = _case(2048, 1024, 48, torch.float32, 1)
    small = _case(128, 96, 10, torch.float64, 2)
    mid = _case(300, 200, 16, torch.bfloat16, 3)
    st, e_big, _, sts = _noalloc(tsk, big[0], big[1], 24, 1)
    assert st == 0 and sts == 0
    for (A, S), r, prec, tol in ((small, 5, 0, 1e-10), (mid, 8, 2, 1e-3), (small, 5, 0, 1e-10)):
        st, e, nrm, sts = _noalloc(tsk, A, S, r, prec)
        assert st == 0 and sts == 0
        o = oracle.scw(A.double().cpu().numpy(), S.double().cpu().numpy(), r, dense=False)
        assert abs(e - o["err"]) <= tol * o["err"], (e, o["err"])
        np.testing.assert_allclose(nrm, o["normA2"], rtol=1e-6)


def test_noalloc_near_exact_matrix_uses_the_direct_error(tsk):
    """A of rank k = r plus noise 1e-6, so S A has full rank and Q spans the
    row space of A's rank-k part: the error is the noise level, the identity
    ||A||^2 - sum sigma^2 cancels, the direct pass takes over, and the error
    matches the oracle's direct ||A - B||_F.  (With rank(A) < k the sketch
    panel would be rank deficient, which the call reports instead.)"""
    g = torch.Generator(device="cpu").manual_seed(9)
    m, n, k, r = 256, 192, 6, 6
    U = torch.linalg.qr(torch.randn(m, k, generator=g, dtype=torch.float64))[0]
    A = U @ torch.randn(k, n, generator=g, dtype=torch.float64) \
        + 1e-6 * torch.randn(m, n, generator=g, dtype=torch.float64)
    S = torch.randn(k, m, generator=g, dtype=torch.float64)
    for dtype, tol in ((torch.float64, 1e-8), (torch.float32, 5e-2)):
        sdt = torch.float64 if dtype == torch.float64 else torch.float32
        Ad, Sd = A.to(dtype).cuda(), S.to(sdt).cuda()
        st, e, _, sts = _noalloc(tsk, Ad, Sd, r, PREC[dtype])
        assert st == 0 and sts == 0
        o = oracle.scw(Ad.double().cpu().numpy(), Sd.double().cpu().numpy(), r, dense=False)
        # the error is about 1e-5 ||A||: the identity alone would leave an
        # error of about sqrt(u) ||A|| (3e-4 ||A|| in FP32, 40 times too big);
        # the direct pass in FP32 is off by the rounding of B, a few percent
        assert abs(e - o["err"]) <= tol * o["err"], (dtype, e, o["err"])


def test_noalloc_reports_a_rank_deficient_sketch(tsk):
    """Two equal sketch rows: rank(SA) = k - 1 < k.  The call itself
    returns TSK_OK (the work is asynchronous) and the status output says
    TSK_ERANKDEF once the work has run; the next call starts clean."""
    rng = np.random.default_rng(5)
    A = torch.tensor(rng.standard_normal((64, 48)), device="cuda")
    S = rng.standard_normal((6, 64))
    S[3] = S[1]
    st, e, _, sts = _noalloc(tsk, A, torch.tensor(S, device="cuda"), 2, 0)
    assert st == 0 and sts == 6
    A2, S2 = _case(128, 96, 10, torch.float64, 4)
    st, e, _, sts = _noalloc(tsk, A2, S2, 5, 0)
    assert st == 0 and sts == 0


def test_noalloc_rejects_sizes_beyond_its_array(tsk):
    lib = tsk.load_library()
    # (m + n) * k_pad * 4 bytes = 70000 * 64 * 4 > 8 MiB; the call is rejected
    # from the sizes alone, before anything reads the (tiny) buffer
    buf = torch.empty(64, device="cuda")
    d = tsk.MatDesc(buf.data_ptr(), buf.data_ptr(), 35000, 35000, 35000, 64, 8)
    err = torch.empty(1, dtype=torch.float64, device="cuda")
    st = lib.tsk_approx_noalloc(C.byref(d), tsk.FP32, C.c_void_p(err.data_ptr()), None,
                                None, None)
    assert st == 1  # TSK_EINVAL, rejected before any device work
    assert b"static array" in lib.tsk_last_error(None)
