"""Two-sided sketching on the GPU against the oracle (Section 3.2).

* Algorithm 3: Q = qr((S A)^T), P = qr(A W^T), the l x k core P^T A Q, its
  rank-r truncation and B = P [P^T A Q]_r Q^T, compared with
  oracle.two_sided_scw on the same S and W: 1e-10 relative in FP64 (errors,
  B), the 1e-3 gap in FP32 / BF16.
* Algorithm 5 (HOOI, HOSVD start): the core energy sum_d ||S A_d W^T||^2 and
  the subspaces of S and W against oracle.hooi.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

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


@pytest.fixture(scope="module")
def c1():
    spec = synth.C1
    tr = synth.stream(spec, "train")
    te = synth.stream(spec, "test")
    S_o, W_o, sweeps = oracle.hooi(list(tr.numpy()), 10, 8)
    return spec, tr, te, S_o, W_o, sweeps


def test_two_sided_scw_fp64_matches_oracle(tsk, c1):
    spec, _, te, S_o, W_o, _ = c1
    h = tsk.Handle()
    out = h.approx_two_sided(te.cuda(), torch.tensor(S_o, device="cuda"),
                             torch.tensor(W_o, device="cuda"), spec.r, outputs=True)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    for i, A in enumerate(te.numpy()):
        o = oracle.two_sided_scw(A, S_o, W_o, spec.r)
        assert abs(float(out["err"][i]) - o["err"]) <= 1e-10 * o["err"], i
        B = _np(out["US"][i]) @ _np(out["Vt"][i])
        assert np.linalg.norm(B - o["B"]) <= 1e-10 * np.linalg.norm(A), i
        np.testing.assert_allclose(_np(out["sigma"][i])[:8], o["core_sigma"][:8], rtol=1e-10,
                                   atol=1e-13 * np.linalg.norm(A))
        np.testing.assert_allclose(float(out["normA2"][i]), float(np.sum(A * A)), rtol=1e-12)
    h.close()


def test_two_sided_ragged_batch_and_edge_shapes(tsk):
    """Different k, l, r per matrix in one call (shared and distinct W),
    l > k, k > l, r = min(k, l), and k = l = 64 (the largest)."""
    rng = np.random.default_rng(17)
    sizes = [(96, 80, 10, 6, 3), (70, 120, 5, 12, 5), (130, 90, 16, 16, 16), (200, 150, 64, 64, 8)]
    As, Ss, Ws, rs = [], [], [], []
    for m, n, k, l, r in sizes:
        As.append(rng.standard_normal((m, n)))
        Ss.append(rng.standard_normal((k, m)))
        Ws.append(rng.standard_normal((l, n)))
        rs.append(r)
    h = tsk.Handle()
    out = h.approx_two_sided([torch.tensor(a, device="cuda") for a in As],
                             [torch.tensor(x, device="cuda") for x in Ss],
                             [torch.tensor(w, device="cuda") for w in Ws], rs)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    for i in range(len(sizes)):
        o = oracle.two_sided_scw(As[i], Ss[i], Ws[i], rs[i])
        assert abs(float(out["err"][i]) - o["err"]) <= 1e-10 * np.linalg.norm(As[i]), i
    h.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_two_sided_reduced_precision(tsk, storage):
    spec = synth.scaled(synth.C2, 320, 264, 24, 6, k=20, r=10, storage=storage)
    tr = synth.stream(spec, "train")
    te = synth.stream(spec, "test")
    S_o, W_o, _ = oracle.hooi(list(tr.double().numpy()), spec.k, spec.k)
    S = torch.tensor(S_o, dtype=torch.float32)
    W = torch.tensor(W_o, dtype=torch.float32)
    h = tsk.Handle()
    out = h.approx_two_sided(te.cuda(), S.cuda(), W.cuda(), spec.r)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    for i, A in enumerate(te.double().numpy()):
        o = oracle.two_sided_scw(A, S.double().numpy(), W.double().numpy(), spec.r)
        assert abs(float(out["err"][i]) - o["err"]) <= GAP * o["err"], i
    h.close()


def test_hooi_fp64_matches_oracle(tsk, c1):
    spec, tr, _, S_o, W_o, sweeps_o = c1
    h = tsk.Handle()
    S, W, energy, sweeps, st = h.train_two_sided(tr.cuda(), 10, 8)
    assert st == 0
    As = list(tr.numpy())
    e_o = sum(float(np.sum((S_o @ A @ W_o.T) ** 2)) for A in As)
    # both stop when a sweep changes the energy by < 1e-12 of sum ||A_d||^2,
    # perhaps one sweep apart: energies agree to about that, subspaces to
    # about its square root
    assert abs(energy - e_o) <= 1e-9 * e_o, (energy, e_o)
    Sg, Wg = _np(S), _np(W)
    assert np.linalg.norm(Sg @ Sg.T - np.eye(10)) < 1e-12
    assert np.linalg.norm(Wg.T @ Wg - W_o.T @ W_o) < 1e-5
    assert np.linalg.norm(Sg.T @ Sg - S_o.T @ S_o) < 1e-5
    assert abs(sweeps - sweeps_o) <= 1
    # the energy of the sketches it returns is the energy it reports
    e_g = sum(float(np.sum((Sg @ A @ Wg.T) ** 2)) for A in As)
    assert abs(e_g - energy) <= 1e-10 * e_g
    h.close()


def test_hooi_reduced_precision(tsk):
    """FP32 and BF16 training matrices: the sketches' Tucker2 energy is
    within 1e-5 of the oracle's converged energy on the same stored values."""
    spec = synth.scaled(synth.C2, 256, 192, 30, 1, k=12, r=6, storage="f32")
    tr = synth.stream(spec, "train")
    for dt in (torch.float32, torch.bfloat16):
        As = list(tr.to(dt).double().numpy())
        S_o, W_o, _ = oracle.hooi(As, 12, 12)
        e_o = sum(float(np.sum((S_o @ A @ W_o.T) ** 2)) for A in As)
        h = tsk.Handle()
        S, W, energy, sweeps, st = h.train_two_sided(tr.to(dt).cuda(), 12, 12)
        assert st == 0
        Qs = np.linalg.qr(_np(S).T)[0]
        Qw = np.linalg.qr(_np(W).T)[0]
        e_g = sum(float(np.sum((Qs.T @ A @ Qw) ** 2)) for A in As)
        assert e_g >= (1 - 1e-5) * e_o, (dt, e_g, e_o)
        assert abs(energy - e_o) <= 1e-5 * e_o, (dt, energy, e_o)
        h.close()
