"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test checks the oracle against something the paper or plain
mathematics fixes: hand-derived worked examples (tests/golden), closed forms
built from a known SVD, brute force on tiny inputs, the paper's identities
and inequalities (Theorems 1 and 2, Eq. A.1, Eq. A.3), its special cases
(identical training matrices; scale invariance) and finite differences.
A dropped term, a sign or index error or a transposed operand anywhere in
the oracle fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _orthonormal(rng, m, k):
    Q, _ = np.linalg.qr(rng.standard_normal((m, k)))
    return Q


def _with_spectrum(rng, m, n, s):
    """A = U diag(s) V^T with random orthonormal U, V (closed-form SVD)."""
    p = len(s)
    U = _orthonormal(rng, m, p)
    V = _orthonormal(rng, n, p)
    return (U * np.asarray(s)) @ V.T, U, V


# ---------------------------------------------------------------- golden ---
def test_golden_scw_hand_examples():
    data = json.load(open(GOLDEN))
    for case in data["scw_cases"]:
        A = np.array(case["A"], float)
        S = np.array(case["S"], float)
        out = oracle.scw(A, S, case["r"])
        k = S.shape[0]
        np.testing.assert_allclose(out["sigma"][:k], case["sigma"], rtol=1e-14,
                                   atol=1e-14, err_msg=case["name"])
        assert abs(out["err"] - case["err"]) < 1e-14, case["name"]
        opt = oracle.optimal_error(A, case["r"])
        assert abs(opt - case["opt_err"]) < 1e-14, case["name"]
        te = oracle.test_error([out["err"]], [opt])
        assert abs(te - case["test_error"]) < 1e-14, case["name"]


def test_golden_sketch_hand_example():
    case = json.load(open(GOLDEN))["sketch_cases"][0]
    As = [np.array(a, float) for a in case["As"]]
    np.testing.assert_allclose(oracle.gram_mode1(As), case["gram_mode1"], atol=0)
    np.testing.assert_allclose(oracle.gram_mode2(As), case["gram_mode2"], atol=0)
    S, W, lam1, lam2 = oracle.train_sketch(As, case["k"], l=1)
    np.testing.assert_allclose(lam1, case["eigenvalues"], rtol=1e-15)
    np.testing.assert_allclose(S, case["S"], rtol=1e-15)
    np.testing.assert_allclose(W, case["W"], rtol=1e-15)
    assert abs(np.trace(oracle.gram_mode1(As)) - case["trace"]) == 0


# ------------------------------------------------------------------ Gram ---
def test_gram_brute_force_triple_loop(rng):
    D, m, n = 3, 4, 5
    As = [rng.standard_normal((m, n)) for _ in range(D)]
    G = [[0.0] * m for _ in range(m)]
    G2 = [[0.0] * n for _ in range(n)]
    for A in As:
        for i, i2, j in itertools.product(range(m), range(m), range(n)):
            G[i][i2] += A[i][j] * A[i2][j]
        for j, j2, i in itertools.product(range(n), range(n), range(m)):
            G2[j][j2] += A[i][j] * A[i][j2]
    np.testing.assert_allclose(oracle.gram_mode1(As), G, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.gram_mode2(As), G2, rtol=1e-13, atol=1e-13)


def test_gram_trace_is_tensor_norm(rng):
    As = [rng.standard_normal((7, 5)) for _ in range(4)]
    fro2 = sum(float(np.sum(A ** 2)) for A in As)
    assert abs(np.trace(oracle.gram_mode1(As)) - fro2) < 1e-12 * fro2
    assert abs(np.trace(oracle.gram_mode2(As)) - fro2) < 1e-12 * fro2


def test_gram_equals_unfolding_product(rng):
    # A_(1) = [A_1 | ... | A_D'] (Section 3.1, Eq. 3.2)
    As = [rng.standard_normal((6, 4)) for _ in range(3)]
    A1 = np.concatenate(As, axis=1)
    ref = np.einsum("ij,kj->ik", A1, A1)
    np.testing.assert_allclose(oracle.gram_mode1(As), ref, rtol=1e-13)


# ---------------------------------------------------------- eigenvectors ---
def test_eig_2x2_closed_form(rng):
    for _ in range(5):
        a, c = rng.uniform(1, 3, 2)
        b = rng.uniform(-1, 1)
        G = np.array([[a, b], [b, c]])
        half = np.hypot((a - c) / 2, b)
        lam_top = (a + c) / 2 + half
        v = np.array([b, lam_top - a])
        if np.linalg.norm(v) < 1e-12:
            v = np.array([lam_top - c, b])
        v /= np.linalg.norm(v)
        if abs(v[1]) > abs(v[0]) and v[1] < 0 or abs(v[0]) >= abs(v[1]) and v[0] < 0:
            v = -v
        S, lam = oracle.leading_eigvecs(G, 1)
        assert abs(lam[0] - lam_top) < 1e-14 * lam_top
        np.testing.assert_allclose(S[0], v, atol=1e-13)


def test_eig_known_spectrum(rng):
    m, k = 12, 4
    U = _orthonormal(rng, m, m)
    lam = np.sort(rng.uniform(1, 10, m))[::-1]
    G = (U * lam) @ U.T
    S, got = oracle.leading_eigvecs(G, k)
    np.testing.assert_allclose(got, lam, rtol=1e-12)
    P_ref = U[:, :k] @ U[:, :k].T
    assert np.linalg.norm(S.T @ S - P_ref) < 1e-12
    assert np.linalg.norm(S @ S.T - np.eye(k)) < 1e-13          # Eq. 3.1 constraint
    assert np.linalg.norm(G @ S.T - S.T * got[:k]) < 1e-12 * lam[0]
    # canonical signs: the largest-magnitude entry of each row is positive
    for row in S:
        assert row[np.argmax(np.abs(row))] > 0


def test_identical_training_recovers_left_subspace(rng):
    # Section 3.1, Analysis: if every training matrix equals A, S spans U_k.
    m, n, k = 20, 15, 5
    s = np.linspace(5, 1, 10)
    A, U, _ = _with_spectrum(rng, m, n, s)
    S, _, lam, _ = oracle.train_sketch([A] * 6, k)
    assert np.linalg.norm(S.T @ S - U[:, :k] @ U[:, :k].T) < 1e-12
    np.testing.assert_allclose(lam[:10], 6 * s ** 2, rtol=1e-12)


def test_scale_invariance(rng):
    # Section 4: the sketch is unchanged when the training data are scaled.
    As = [rng.standard_normal((10, 8)) for _ in range(5)]
    S1, _, _, _ = oracle.train_sketch(As, 3)
    S2, _, _, _ = oracle.train_sketch([37.5 * A for A in As], 3)
    np.testing.assert_allclose(S1, S2, atol=1e-13)


def test_sketch_maximises_captured_energy(rng):
    # Eq. 3.2: S* maximises sum_d ||S A_d||_F^2 over row-orthonormal S.
    As = [rng.standard_normal((9, 7)) for _ in range(4)]
    S, _, lam, _ = oracle.train_sketch(As, 3)
    best = sum(float(np.sum((S @ A) ** 2)) for A in As)
    assert abs(best - lam[:3].sum()) < 1e-12 * best
    for _ in range(20):
        R = _orthonormal(rng, 9, 3).T
        assert sum(float(np.sum((R @ A) ** 2)) for A in As) <= best + 1e-12


# ------------------------------------------------------------------- SCW ---
def test_optimal_error_closed_form(rng):
    s = np.array([9.0, 5.0, 3.0, 2.0, 1.0, 0.5])
    A, _, _ = _with_spectrum(rng, 15, 11, s)
    for r in range(1, 6):
        assert abs(oracle.optimal_error(A, r) - np.sqrt(np.sum(s[r:] ** 2))) < 1e-13


def test_eckart_young_lower_bound(rng):
    for _ in range(10):
        A = rng.standard_normal((14, 10))
        S = rng.standard_normal((4, 14))
        out = oracle.scw(A, S, 2)
        assert out["err"] >= oracle.optimal_error(A, 2) * (1 - 1e-13)


def test_full_sketch_recovers_optimum(rng):
    # k = m with an invertible S: the row space of SA is that of A.
    m, n, r = 8, 11, 3
    A = rng.standard_normal((m, n))
    S = rng.standard_normal((m, m))
    out = oracle.scw(A, S, r)
    assert abs(out["err"] - oracle.optimal_error(A, r)) < 1e-12 * np.linalg.norm(A)
    # and with k = n when m > n (every sketch then spans R^n)
    A = rng.standard_normal((12, 7))
    S = rng.standard_normal((7, 12))
    out = oracle.scw(A, S, r)
    assert abs(out["err"] - oracle.optimal_error(A, r)) < 1e-12 * np.linalg.norm(A)


def test_exact_left_subspace_sketch_is_optimal(rng):
    s = np.array([6.0, 4.0, 3.0, 1.0, 0.7, 0.2, 0.1])
    A, U, _ = _with_spectrum(rng, 16, 12, s)
    for k, r in [(3, 2), (5, 3), (4, 4)]:
        S = U[:, :k].T
        out = oracle.scw(A, S, r)
        assert abs(out["err"] - np.sqrt(np.sum(s[r:] ** 2))) < 1e-12
        np.testing.assert_allclose(out["sigma"], s[:k], rtol=1e-12)


def test_exact_recovery_from_training(rng):
    # Every stream matrix lies in the column space of U0 (rank L <= k).
    m, n, L, k = 24, 18, 4, 6
    U0 = _orthonormal(rng, m, L)
    train = [U0 @ rng.standard_normal((L, n)) for _ in range(10)]
    S, _, _, _ = oracle.train_sketch(train, k)
    A = U0 @ rng.standard_normal((L, n))
    for r in (2, 4):
        out = oracle.scw(A, S, r)
        assert abs(out["err"] - oracle.optimal_error(A, r)) < 1e-12 * np.linalg.norm(A)
    assert oracle.scw(A, S, L)["err"] < 1e-12 * np.linalg.norm(A)


def test_projection_identity(rng):
    # Eq. A.3: ||A - [AQ]_r Q^T||^2 = ||A||^2 - ||[AQ]_r||^2.
    for _ in range(5):
        A = rng.standard_normal((13, 9))
        S = rng.standard_normal((5, 13))
        out = oracle.scw(A, S, 3)
        ident = out["normA2"] - np.sum(out["sigma"][:3] ** 2)
        assert abs(out["err"] ** 2 - ident) < 1e-12 * out["normA2"]
        B = out["US"] @ out["Vt"]
        np.testing.assert_allclose(B, out["B"], atol=1e-13)
        # Vt rows are orthonormal (Q V_r with Q, V_r orthonormal)
        assert np.linalg.norm(out["Vt"] @ out["Vt"].T - np.eye(3)) < 1e-13


def test_sketch_identity(rng):
    # Section 3.1: ||A - S^T S A||^2 = ||A||^2 - ||SA||^2 for row-orthonormal S.
    A = rng.standard_normal((10, 8))
    S = _orthonormal(rng, 10, 4).T
    lhs = np.sum((A - S.T @ S @ A) ** 2)
    assert abs(lhs - (np.sum(A ** 2) - np.sum((S @ A) ** 2))) < 1e-12


def test_svd_and_qr_forms_agree(rng):
    # Section 3.2: the SVD in line 1 of Algorithm 1 may be replaced by QR.
    for _ in range(5):
        A = rng.standard_normal((11, 9))
        S = rng.standard_normal((5, 11))
        B_svd = oracle.scw_svd_form(A, S, 3)
        np.testing.assert_allclose(oracle.scw(A, S, 3)["B"], B_svd, atol=1e-12)


def test_intermediate_bound_A1(rng):
    # Eq. A.1 per matrix: ||A - SCW||^2 <= ||A - S^T [SA]_r||^2.
    for _ in range(10):
        A = rng.standard_normal((12, 10))
        S = _orthonormal(rng, 12, 5).T
        U, s, Vh = np.linalg.svd(S @ A, full_matrices=False)
        SAr = (U[:, :2] * s[:2]) @ Vh[:2]
        rhs = np.sum((A - S.T @ SAr) ** 2)
        assert oracle.scw(A, S, 2)["err"] ** 2 <= rhs * (1 + 1e-12)


def test_theorem_1(rng):
    # Eq. 3.4 with the trained S: sum_d err_d^2 <= ||calA||^2 - ||[S A_(1)]_r||^2
    m, n, D, k, r = 16, 12, 8, 5, 2
    U0 = _orthonormal(rng, m, 6)
    As = [U0 @ rng.standard_normal((6, n)) + 0.1 * rng.standard_normal((m, n))
          for _ in range(D)]
    S, _, lam, _ = oracle.train_sketch(As, k)
    lhs = sum(oracle.scw(A, S, r)["err"] ** 2 for A in As)
    fro2 = sum(np.sum(A ** 2) for A in As)
    rhs = fro2 - lam[:r].sum()
    A1 = np.concatenate(As, axis=1)
    sv = np.linalg.svd(S @ A1, compute_uv=False)
    assert abs(lam[:r].sum() - np.sum(sv[:r] ** 2)) < 1e-10 * fro2
    assert lhs <= rhs * (1 + 1e-12)
    # and for a random row-orthonormal S as well
    R = _orthonormal(rng, m, k).T
    lhs = sum(oracle.scw(A, R, r)["err"] ** 2 for A in As)
    sv = np.linalg.svd(R @ A1, compute_uv=False)
    assert lhs <= (fro2 - np.sum(sv[:r] ** 2)) * (1 + 1e-12)


def test_theorem_2(rng):
    # Eq. 3.5 (bound of its proof): err^2 - opt^2 <= ||U_k U_k^T - S^T S||_2^2 ||A||_F^2
    s = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.3, 0.1])
    A, U, _ = _with_spectrum(rng, 18, 14, s)
    k, r = 4, 2
    for eps in (1e-3, 1e-2, 0.1, 0.5):
        P = _orthonormal(rng, 18, k)
        S = np.linalg.qr(U[:, :k] + eps * P)[0].T
        err2 = oracle.scw(A, S, r)["err"] ** 2
        opt2 = oracle.optimal_error(A, r) ** 2
        gap = np.linalg.norm(U[:, :k] @ U[:, :k].T - S.T @ S, 2)
        assert err2 - opt2 <= gap ** 2 * np.sum(A ** 2) + 1e-12


def test_scw_batch_coordinate_sketch_closed_form():
    """Problem 1.1 per matrix, in batch order.  With S = the first k rows of
    the identity and a diagonal A, S A keeps the first k rows, so Q spans
    e_1 .. e_k, A Q holds a_1 .. a_k on its diagonal and [A Q]_r keeps the r
    largest of them: err^2 = ||A||^2 - (sum of the r largest a_i^2, i <= k).
    Three matrices with different diagonals (one with its largest entries
    outside the first k) must come back in order; an empty batch gives an
    empty list."""
    n, k, r = 7, 4, 2
    diags = [np.array([5.0, 1.0, 3.0, 2.0, 0.5, 0.25, 0.1]),
             np.array([0.2, 0.3, 0.1, 0.4, 9.0, 8.0, 7.0]),
             np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0])]
    S = np.eye(n)[:k]
    errs = oracle.scw_batch([np.diag(d) for d in diags], S, r)
    assert len(errs) == 3
    for e, d in zip(errs, diags):
        top = np.sort(d[:k] ** 2)[::-1][:r].sum()
        assert e == pytest.approx(np.sqrt(np.sum(d ** 2) - top), rel=1e-12)
    assert oracle.scw_batch([], S, r) == []


def test_test_error_definition():
    # Eq. 4.1 on numbers checked by hand: mean of (1.1-1)/1 and (2.4-2)/2.
    assert abs(oracle.test_error([1.1, 2.4], [1.0, 2.0]) - 0.15) < 1e-15


# --------------------------------------------------------------- refiner ---
def test_refiner_loss_matches_scw(rng):
    As = [rng.standard_normal((10, 8)) for _ in range(3)]
    S = rng.standard_normal((4, 10))
    expect = np.mean([oracle.scw(A, S, 2)["err"] ** 2 / np.sum(A ** 2) for A in As])
    assert abs(oracle.ivy_loss(S, As, 2) - expect) < 1e-14


def test_refiner_gradient_finite_differences(rng):
    m, n, k, r = 14, 11, 5, 2
    U0 = _orthonormal(rng, m, 6)
    As = [U0 @ np.diag([4, 3, 2, 1, .5, .2]) @ rng.standard_normal((6, n))
          + 0.05 * rng.standard_normal((m, n)) for _ in range(3)]
    S = rng.standard_normal((k, m))
    g = oracle.ivy_grad(S, As, r)
    h = 1e-6 * np.linalg.norm(S)
    for _ in range(20):
        Dd = rng.standard_normal(S.shape)
        Dd /= np.linalg.norm(Dd)
        fd = (oracle.ivy_loss(S + h * Dd, As, r) - oracle.ivy_loss(S - h * Dd, As, r)) / (2 * h)
        an = float(np.sum(g * Dd))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), np.linalg.norm(g) * 1e-3) + 1e-10


# ------------------------------------------------------------- two-sided ---
def test_two_sided_with_identity_W_is_one_sided(rng):
    A = rng.standard_normal((12, 8))
    S = rng.standard_normal((4, 12))
    W = np.eye(8)
    assert abs(oracle.two_sided_scw(A, S, W, 2)["err"]
               - oracle.scw(A, S, 2)["err"]) < 1e-12


def test_hooi_exact_tucker2_recovery(rng):
    m, n, D, k, l = 12, 10, 6, 3, 2
    U = _orthonormal(rng, m, k)
    V = _orthonormal(rng, n, l)
    As = [U @ rng.standard_normal((k, l)) @ V.T for _ in range(D)]
    S, W, _ = oracle.hooi(As, k, l)
    assert np.linalg.norm(S.T @ S - U @ U.T) < 1e-10
    assert np.linalg.norm(W.T @ W - V @ V.T) < 1e-10
    for A in As:
        assert oracle.two_sided_scw(A, S, W, min(k, l))["err"] < 1e-10 * np.linalg.norm(A)


def test_hooi_core_energy_monotone(rng):
    As = [rng.standard_normal((9, 8)) for _ in range(5)]
    energies = []
    for sweeps in (1, 2, 3, 5):
        S, W, _ = oracle.hooi(As, 3, 3, max_sweeps=sweeps, tol=0.0)
        energies.append(sum(np.sum((S @ A @ W.T) ** 2) for A in As))
    assert all(b >= a - 1e-10 for a, b in zip(energies, energies[1:]))
