"""The tcgen05/TMA BF16 sketch kernel against the oracle and the SIMT path.

Cluster sizes follow m (512 rows per CTA): m <= 512 runs on single CTAs,
m <= 1024 on pairs, m <= 2048 on clusters of 4 and m <= 4096 on clusters of
8.  Ragged n exercises partial 64-column blocks; ragged m exercises rows
past the end of the matrix inside a CTA's slice.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
GAP = 1e-3


@pytest.fixture(scope="module")
def tsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2209_14637_gb300 as mod
    from paper_2209_14637_gb300 import build
    build.build()
    return mod


def _np(t):
    return t.detach().double().cpu().numpy()


def _case(m, n, k, seed, low_rank=True):
    g = torch.Generator(device="cuda").manual_seed(seed)
    if low_rank:
        L = min(2 * k, m, n)
        U = torch.linalg.qr(torch.randn(m, L, generator=g, device="cuda"))[0]
        sv = torch.arange(1, L + 1, device="cuda", dtype=torch.float32) ** -1.2
        A = (U * sv) @ torch.randn(L, n, generator=g, device="cuda") \
            + 1e-3 * torch.randn(m, n, generator=g, device="cuda")
        S = torch.linalg.qr(U[:, :k] + 0.1 * torch.randn(m, k, generator=g, device="cuda"))[0].T
    else:
        A = torch.randn(m, n, generator=g, device="cuda")
        S = torch.randn(k, m, generator=g, device="cuda")
    return A.to(torch.bfloat16).contiguous(), S.contiguous()


def _run(tsk, kernel, As, Ss, rs, outputs=True):
    h = tsk.Handle(kernel=kernel)
    out = h.approx_batch(As, Ss, rs, outputs=outputs)
    torch.cuda.synchronize()
    st = h.sync_status()
    return out, st, h


def test_tc_small_single_cta(tsk):
    A, S = _case(256, 192, 16, 1)
    out, st, h = _run(tsk, tsk.KERNEL_TC, [A], [S], [8])
    assert st == 0
    o = oracle.scw(_np(A), _np(S), 8)
    assert abs(float(out["err"][0]) - o["err"]) <= GAP * o["err"]
    np.testing.assert_allclose(_np(out["normA2"])[0], o["normA2"], rtol=1e-6)
    np.testing.assert_allclose(_np(out["sigma"][0])[:8], o["sigma"][:8], rtol=1e-3)
    h.close()


@pytest.mark.parametrize("m,n,k,r", [
    (512, 200, 20, 10),     # 1 CTA of 512 rows, ragged n
    (1000, 448, 40, 20),    # 2 CTAs of 512 rows, ragged m
    (2048, 576, 40, 20),    # 4 CTAs of 512 rows
    (3000, 136, 10, 5),     # 8 CTAs of 512 rows, ragged m and n
    (300, 72, 48, 24),      # k = 48 (largest the kernel takes)
])
def test_tc_matches_oracle(tsk, m, n, k, r):
    A, S = _case(m, n, k, m + n)
    out, st, h = _run(tsk, tsk.KERNEL_TC, [A], [S], [r])
    assert st == 0
    o = oracle.scw(_np(A), _np(S), r)
    gap = abs(float(out["err"][0]) - o["err"]) / o["err"]
    assert gap <= GAP, gap
    np.testing.assert_allclose(_np(out["normA2"])[0], o["normA2"], rtol=1e-6)
    B = _np(out["US"][0]) @ _np(out["Vt"][0])
    assert np.linalg.norm(B - o["B"]) <= 2e-2 * np.linalg.norm(o["B"])
    h.close()


def test_tc_ragged_batch_matches_simt(tsk):
    sizes = [(256, 256, 10), (700, 320, 20), (1536, 640, 40), (4096, 256, 40),
             (520, 1000, 20), (2048, 2048, 40), (128, 64, 10)]
    As, Ss, rs = [], [], []
    for i, (m, n, k) in enumerate(sizes):
        A, S = _case(m, n, k, 100 + i)
        As.append(A)
        Ss.append(S)
        rs.append(k // 2)
    tc, st, h1 = _run(tsk, tsk.KERNEL_TC, As, Ss, rs, outputs=False)
    assert st == 0
    simt, st2, h2 = _run(tsk, tsk.KERNEL_SIMT, As, Ss, rs, outputs=False)
    assert st2 == 0
    for i in range(len(sizes)):
        o = oracle.scw(_np(As[i]), _np(Ss[i]), rs[i], dense=False)
        assert abs(float(tc["err"][i]) - o["err"]) <= GAP * o["err"], i
        assert abs(float(simt["err"][i]) - o["err"]) <= GAP * o["err"], i
    np.testing.assert_allclose(_np(tc["normA2"]), _np(simt["normA2"]), rtol=1e-5)
    h1.close()
    h2.close()


def test_tc_rejects_unaligned_rows(tsk):
    # a row of 70 BF16 values is 140 bytes: not a multiple of 16, so TMA
    # cannot tile it; asking for the tensor-core kernel explicitly fails
    A, S = _case(128, 70, 8, 3)
    h = tsk.Handle(kernel=tsk.KERNEL_TC)
    with pytest.raises(tsk.TskError) as e:
        h.approx_batch([A], [S], 4)
    assert e.value.status == 7  # TSK_EUNSUPPORTED
    h.close()
    # the automatic choice falls back to the CUDA-core kernels
    out, st, h = _run(tsk, tsk.KERNEL_AUTO, [A], [S], [4])
    o = oracle.scw(_np(A), _np(S), 4, dense=False)
    assert st == 0 and abs(float(out["err"][0]) - o["err"]) <= GAP * o["err"]
    h.close()


def test_tc_repeated_plan_is_deterministic(tsk):
    A, S = _case(2048, 512, 40, 7)
    h = tsk.Handle(kernel=tsk.KERNEL_TC)
    As = [A] * 9
    err = torch.empty(9, dtype=torch.float64, device="cuda")
    plan = h.plan(As, S, 20, err)
    plan.execute()
    first = err.clone()
    for _ in range(3):
        plan.execute()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    # ||A||^2 is summed with atomics, so only the last bits may differ
    assert torch.allclose(first, err, rtol=1e-12, atol=0)
    assert torch.allclose(err, err[0].expand(9), rtol=1e-12, atol=0)
    plan.close()
    h.close()
