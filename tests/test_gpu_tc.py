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


def test_unaligned_rows_are_copied_for_the_tensor_cores(tsk):
    """A row of 70 BF16 values is 140 bytes, not a multiple of 16, so TMA
    cannot tile it: the plan copies A to rows of 72 elements in its
    workspace and the tensor-core kernel reads the copy (TSK_KERNEL_TC
    accepts it); the error matches the oracle and the CUDA-core kernels,
    also for an A that starts off a 16-byte boundary."""
    A, S = _case(128, 70, 8, 3)
    buf = torch.zeros(128 * 70 + 3, dtype=torch.bfloat16, device="cuda")
    buf[3:].view(128, 70).copy_(A)
    A_off = buf[3:].view(128, 70)  # starts 6 bytes past a 16-byte boundary
    assert A_off.data_ptr() % 16 != 0
    o = oracle.scw(_np(A), _np(S), 4, dense=False)
    for Ax in (A, A_off):
        for kern in (tsk.KERNEL_TC, tsk.KERNEL_AUTO, tsk.KERNEL_SIMT):
            out, st, h = _run(tsk, kern, [Ax], [S], [4])
            assert st == 0, kern
            assert abs(float(out["err"][0]) - o["err"]) <= GAP * o["err"], kern
            np.testing.assert_allclose(float(out["normA2"][0]), o["normA2"], rtol=1e-6)
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


def _errs(tsk, refine, As, Ss, rs, kernel=None):
    h = tsk.Handle(kernel=tsk.KERNEL_TC if kernel is None else kernel, refine_q=refine)
    out = h.approx_batch(As, Ss, rs)
    torch.cuda.synchronize()
    st = h.sync_status()
    h.close()
    return _np(out["err"]), st


def test_refinement_modes_on_a_stream_sample(tsk):
    """C3-shaped stream (k = 40, r = 20; 1024 x 1024): every refinement mode
    meets the gap; the automatic mode takes each matrix either unrefined or
    refined, bit for bit like the fixed modes (the same arithmetic in the
    same order), and on this well-conditioned stream leaves all unrefined."""
    import synth
    spec = synth.scaled(synth.C3, 1024, 1024, 24, 6)
    tr = synth.stream(spec, "train")
    S_o, _, _, _ = oracle.train_sketch(list(tr.double().numpy()), spec.k)
    te = synth.stream(spec, "test", device="cuda")
    S = torch.tensor(S_o, device="cuda", dtype=torch.float32)
    As, Ss, rs = list(te), [S] * len(te), [spec.r] * len(te)
    e0, s0 = _errs(tsk, tsk.REFINE_NEVER, As, Ss, rs)
    e1, s1 = _errs(tsk, tsk.REFINE_ALWAYS, As, Ss, rs)
    e2, s2 = _errs(tsk, tsk.REFINE_AUTO, As, Ss, rs)
    assert s0 == s1 == s2 == 0
    ref = np.array([oracle.scw(_np(A), S_o.astype(np.float32).astype(np.float64), spec.r,
                               dense=False)["err"] for A in As])
    for e in (e0, e1, e2):
        assert np.max(np.abs(e - ref) / ref) <= GAP
    assert np.array_equal(e2, e0)


def test_automatic_refinement_where_the_bound_asks(tsk):
    """Two nearly parallel sketch rows make X ill conditioned along one
    direction: the first-order bound exceeds 1e-3 of the residual, so the
    automatic mode refines every matrix (bit for bit the always-refine
    result) and stays within the gap.  FP32 inputs (CUDA-core sketch): the
    BF16 path rounds S to BF16, a relative perturbation of 2^-9 that such a
    sketch amplifies past the gap by itself."""
    g = torch.Generator(device="cuda").manual_seed(11)
    m, n, k, r = 1024, 768, 40, 20
    L = 2 * k
    U = torch.linalg.qr(torch.randn(m, L, generator=g, device="cuda"))[0]
    sv = torch.arange(1, L + 1, device="cuda", dtype=torch.float32) ** -1.2
    As = [((U * sv) @ torch.randn(L, n, generator=g, device="cuda")
           + 1e-3 * torch.randn(m, n, generator=g, device="cuda")).contiguous()
          for _ in range(4)]
    S = torch.linalg.qr(U[:, :k] + 0.1 * torch.randn(m, k, generator=g, device="cuda"))[0].T
    S = S.contiguous()
    S[5] = S[3] + 0.02 * torch.randn(m, generator=g, device="cuda") / m ** 0.5
    Ss, rs = [S] * len(As), [r] * len(As)
    e1, s1 = _errs(tsk, tsk.REFINE_ALWAYS, As, Ss, rs, kernel=tsk.KERNEL_AUTO)
    e2, s2 = _errs(tsk, tsk.REFINE_AUTO, As, Ss, rs, kernel=tsk.KERNEL_AUTO)
    assert s1 == s2 == 0
    assert np.array_equal(e2, e1)
    Sn = _np(S)
    ref = np.array([oracle.scw(_np(A), Sn, r, dense=False)["err"] for A in As])
    assert np.max(np.abs(e2 - ref) / ref) <= GAP


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("m,n,D", [(320, 200, 11), (2048, 256, 20), (128, 64, 3),
                                   (300, 72, 40), (4096, 64, 3)])
def test_tc_gram_mode1(tsk, m, n, D, tile):
    """T1 on the tensor cores (BF16, mode 1) against the FP64 oracle on the
    same stored values, with 256 x 256 tiles on CTA pairs (tile 0) and
    128 x 128 tiles on single CTAs (tile 1): ragged m (partial tiles, and a
    pair whose second CTA holds only rows past m) and n (a partial 64-column
    block), matrices split over CTAs (FP64 atomics) or not, more than two
    TMEM flush groups of eight matrices, and m = 4096 (more tiles than
    SMs)."""
    g = torch.Generator(device="cuda").manual_seed(m + n + D)
    T = [torch.randn(m, n, generator=g, device="cuda").to(torch.bfloat16) for _ in range(D)]
    h = tsk.Handle(gram_tile=tile)
    G = _np(h.gram(T, mode=1))
    assert h.sync_status() == 0
    R = oracle.gram_mode1([_np(t) for t in T])
    _gram_entrywise(G, R, 1e-5)
    assert np.array_equal(G, G.T)
    Gs = h.gram(T[:2], mode=1)
    h.gram(T[2:], mode=1, out=Gs, accumulate=True)
    _gram_entrywise(_np(Gs), R, 1e-5)
    h.close()


@pytest.mark.parametrize("tile", [0, 1])
@pytest.mark.parametrize("m,n,D", [(200, 320, 11), (2048, 256, 20), (64, 128, 3),
                                   (72, 300, 40), (96, 2048, 3)])
def test_tc_gram_mode2(tsk, m, n, D, tile):
    """T1' on the tensor cores: G2 = sum A_d^T A_d (n x n) with MN-major
    operands (columns of A along M, rows along K) against the FP64 oracle
    on the same stored values, entrywise, on 256 x 256 tiles of CTA pairs
    (tile 0) and 128 x 128 tiles of single CTAs (tile 1): ragged n (partial
    tiles, pairs whose second CTA holds only columns past n) and m (a
    partial 64-row K slice), splits over CTAs or not, several flush groups,
    n = 2048 (many tiles)."""
    g = torch.Generator(device="cuda").manual_seed(7 * m + n + D)
    T = [torch.randn(m, n, generator=g, device="cuda").to(torch.bfloat16) for _ in range(D)]
    h = tsk.Handle(gram_tile=tile)
    G = _np(h.gram(T, mode=2))
    assert h.sync_status() == 0
    R = oracle.gram_mode2([_np(t) for t in T])
    _gram_entrywise(G, R, 1e-5)
    assert np.array_equal(G, G.T)
    Gs = h.gram(T[:2], mode=2)
    h.gram(T[2:], mode=2, out=Gs, accumulate=True)
    _gram_entrywise(_np(Gs), R, 1e-5)
    h.close()


def _gram_entrywise(G, R, tol):
    """|G_ij - R_ij| <= tol sqrt(R_ii R_jj) for every entry (Cauchy-Schwarz
    scale of the entry)."""
    d = np.sqrt(np.clip(np.diag(R), 0.0, None))
    worst = np.max(np.abs(G - R) / (tol * np.outer(d, d) + 1e-300))
    assert worst <= 1.0, worst


def test_mixed_batch_routes_by_k_and_copies_unaligned_rows(tsk):
    """A BF16 batch with rows TMA cannot move as they are (2n not a multiple
    of 16 bytes: copied to aligned rows, then the tensor-core kernel),
    aligned rows (tensor-core kernel directly) and k = 56 > 48 (CUDA-core
    kernels), in one plan (217 x 181 is the MRI slice shape, below the C4
    size range): every error, ||A||^2 and factor matches the oracle, and
    asking for the tensor-core kernel alone is refused because of the
    k = 56 matrix only."""
    sizes = [(300, 77, 16), (512, 200, 20), (257, 131, 10), (1024, 64, 40),
             (129, 333, 12), (700, 520, 24), (217, 181, 20), (400, 300, 56)]
    As, Ss, rs = [], [], []
    for i, (m, n, k) in enumerate(sizes):
        A, S = _case(m, n, k, 500 + i)
        As.append(A)
        Ss.append(S)
        rs.append(k // 2)
    out, st, h = _run(tsk, tsk.KERNEL_AUTO, As, Ss, rs)
    assert st == 0
    for i in range(len(sizes)):
        o = oracle.scw(_np(As[i]), _np(Ss[i]), rs[i])
        assert abs(float(out["err"][i]) - o["err"]) <= GAP * o["err"], i
        np.testing.assert_allclose(_np(out["normA2"])[i], o["normA2"], rtol=1e-6)
        B = _np(out["US"][i]) @ _np(out["Vt"][i])
        assert np.linalg.norm(B - o["B"]) <= 2e-2 * np.linalg.norm(o["B"]), i
    h.close()
    h2 = tsk.Handle(kernel=tsk.KERNEL_TC)
    with pytest.raises(tsk.TskError) as e:
        h2.approx_batch(As, Ss, rs)
    assert e.value.status == 7
    out2 = h2.approx_batch(As[:-1], Ss[:-1], rs[:-1])  # without k = 56
    torch.cuda.synchronize()
    assert h2.sync_status() == 0
    np.testing.assert_allclose(_np(out2["err"]), _np(out["err"])[:-1], rtol=1e-12)
    h2.close()


def test_padded_rows_take_the_tensor_cores(tsk):
    """Unaligned widths stored with a padded leading dimension (a multiple
    of 8 elements) go to the tensor-core kernel: it runs alone (TSK_KERNEL_TC
    accepts the batch) and matches the oracle."""
    sizes = [(300, 77, 16), (257, 131, 10), (1500, 333, 40)]
    As, Ss, rs = [], [], []
    for i, (m, n, k) in enumerate(sizes):
        A, S = _case(m, n, k, 700 + i)
        ld = (n + 7) // 8 * 8
        buf = torch.zeros(m, ld, dtype=torch.bfloat16, device="cuda")
        buf[:, :n] = A
        As.append(buf[:, :n])
        Ss.append(S)
        rs.append(k // 2)
    out, st, h = _run(tsk, tsk.KERNEL_TC, As, Ss, rs)
    assert st == 0
    for i in range(len(sizes)):
        o = oracle.scw(_np(As[i]), _np(Ss[i]), rs[i], dense=False)
        assert abs(float(out["err"][i]) - o["err"]) <= GAP * o["err"], i
    h.close()



@pytest.mark.parametrize("m,n,k", [(300, 200, 16), (700, 136, 40), (1000, 448, 24),
                                   (2048, 576, 40), (2200, 104, 10)])
def test_tc_384_row_ctas(tsk, tmp_path, m, n, k):
    """The 384-row shape (three stages of A; clusters of 1, 2, 3 and 6 CTAs,
    rows of X~ padded to a multiple the cluster size divides, an S image of
    round8(k) rows) chosen through a tuning table, against the oracle."""
    import json
    c512 = 1
    while c512 * 512 < m:
        c512 *= 2
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"kernel": "sketch_tc", "classes": [
        {"cluster_at_512": c512, "k8": (k + 7) // 8 * 8, "rows_per_cta": 384}]}))
    A, S = _case(m, n, k, 900 + m)
    h = tsk.Handle(kernel=tsk.KERNEL_TC)
    h.autotune_load(str(path))
    out = h.approx_batch([A], [S], k // 2, outputs=True)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    o = oracle.scw(_np(A), _np(S), k // 2)
    assert abs(float(out["err"][0]) - o["err"]) <= GAP * o["err"]
    np.testing.assert_allclose(_np(out["normA2"])[0], o["normA2"], rtol=1e-6)
    B = _np(out["US"][0]) @ _np(out["Vt"][0])
    assert np.linalg.norm(B - o["B"]) <= 2e-2 * np.linalg.norm(o["B"])
    h.close()


def test_expired_waits_report_a_timeout_and_leave_the_context_usable(tsk):
    """Failure detection without a fault: a spin limit of one iteration
    (120 ns) makes the single-CTA tensor-core kernel's bounded waits run out
    while its loads are still in flight.  The kernel raises the timeout bit,
    stops issuing and stops arriving on barriers whose phases can no longer
    complete, drains its own loads and tensor-core operations (those drains
    have their own two-second bound), frees its TMEM and returns: the host
    reads TSK_ETIMEOUT, and a normal handle then runs the same case
    correctly on the same context."""
    A, S = _case(384, 256, 16, 21)  # m <= 512: one CTA, no peers in a cluster
    h = tsk.Handle(kernel=tsk.KERNEL_TC, spin_limit=1)
    h.approx_batch([A], [S], 8)
    assert h.sync_status() == 5  # TSK_ETIMEOUT
    assert h.sync_status() == 0  # read and cleared
    h.close()
    out, st, h2 = _run(tsk, tsk.KERNEL_TC, [A], [S], [8])
    assert st == 0
    o = oracle.scw(_np(A), _np(S), 8, dense=False)
    assert abs(float(out["err"][0]) - o["err"]) <= GAP * o["err"]
    h2.close()


@pytest.mark.parametrize("m,n,D,dtype,lda", [
    (320, 200, 11, torch.bfloat16, 200),   # 16-byte rows: vector loads
    (2048, 256, 20, torch.bfloat16, 256),
    (130, 64, 3, torch.bfloat16, 64),
    (150, 100, 9, torch.bfloat16, 100),    # 200-byte rows: scalar loads
    (96, 203, 10, torch.float32, 208),     # FP32, padded rows: vectors and a 3-wide tail
    (64, 77, 17, torch.float32, 77),       # FP32, scalar
])
def test_e4m3_quantization_and_gram(tsk, m, n, D, dtype, lda):
    """FP8 training Gram: the quantizer's scales and bytes equal the oracle's
    bit for bit (per (group of eight, row) the smallest power of two
    s >= 2^-149 with max |A| <= 448 s, s = 1 for a zero row; each byte the
    E4M3 rounding, to nearest even, of A / s).  Edge rows: maxima of exactly
    448 (s = 1) and 896 (s = 2), a zero row, and a row at 2^-130 (s = 2^-138,
    whose reciprocal leaves FP32's range).  The tensor-core Gram of the E4M3
    copies (kind::f8f6f4 on CTA pairs) equals the oracle's FP64 Gram of the
    values they stand for, entrywise."""
    g = torch.Generator(device="cuda").manual_seed(m + 3 * n + D)
    rows = torch.logspace(-3, 3, m, device="cuda")[:, None]  # rows of very unequal size
    buf = torch.randn(D, m, lda, generator=g, device="cuda") * rows
    buf[:, 0] = buf[:, 0].clamp(-400, 400)
    buf[:, 0, 0] = 448.0
    buf[:, 1] = buf[:, 1].clamp(-800, 800)
    buf[:, 1, n - 1] = -896.0
    buf[:, 2] = 0.0
    buf[:, 3] = buf[:, 3].clamp(-1.9, 1.9) * 2.0 ** -131
    buf[:, 3, n // 2] = 2.0 ** -130
    buf = buf.to(dtype)
    T = [buf[d, :, :n] for d in range(D)]
    h = tsk.Handle()
    A8, scales = h.quantize_e4m3(T)
    torch.cuda.synchronize()
    codes_o, scales_o = oracle.quantize_e4m3([t.double().cpu().numpy() for t in T])
    assert np.array_equal(scales.cpu().double().numpy(), scales_o)
    assert scales_o[0, 0] == 1.0 and scales_o[0, 1] == 2.0 and scales_o[0, 2] == 1.0
    assert scales_o[0, 3] == 2.0 ** -138
    assert np.array_equal(A8[:, :, :n].cpu().numpy(), codes_o)
    G = _np(h.gram_e4m3(A8, scales, n))
    assert h.sync_status() == 0
    R = oracle.gram_mode1(list(oracle.dequantize_e4m3(codes_o, scales_o)))
    _gram_entrywise(G, R, 1e-5)
    assert np.array_equal(G, G.T)
    h.close()
