"""Test side of the method, in float64 (test infrastructure).

Algorithm 1 (SCW): with V^T from the SVD of SA, take [AV]_r, the truncated
rank-r SVD of AV, and return [AV]_r V^T.  The paper notes (Section 3.2,
two-sided SCW paragraph) that the SVD in line 1 only orthogonalises the row
space of SA and may be replaced by a QR decomposition; the proof of
Theorem 1 uses exactly that: Q (n x k) column-orthonormal in the row space
of SA.  scw() follows that QR form; scw_svd_form() is the literal thin-SVD
form and serves to pin the two against each other.

Reading of "full SVD of SA" (Algorithm 1, line 1): a full SVD would give an
n x n V and make AV = A, so the thin SVD (V n x k) is meant, matching
"Q in R^{n x k}" in the proof of Theorem 1.
"""
from __future__ import annotations

import numpy as np


def _thin_qr(X: np.ndarray):
    Q, R = np.linalg.qr(X, mode="reduced")
    return Q, R


def scw(A, S, r: int, dense: bool = True):
    """SCW(A, S, r) in the QR form (Algorithm 1 with the Section 3.2 remark).

    Steps, in the paper's order:
      1. X = (S A)^T (n x k); Q, R = thin QR of X   (Algorithm 3, line 1)
      2. M = A Q (m x k); U, s, Vh = thin SVD of M; keep the top r
         ([AQ]_r, Algorithm 1, line 2)
      3. B = [AQ]_r Q^T = (U_r s_r) (Q V_r)^T       (Algorithm 1, line 3)
      4. err = ||A - B||_F, computed elementwise    (problem 1.1)

    Returns a dict with US = U_r diag(s_r) (m x r), Vt = (Q V_r)^T (r x n),
    sigma (k singular values of AQ, descending), err, normA2 = ||A||_F^2,
    and B (dense, if requested).
    """
    A = np.asarray(A, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    k = S.shape[0]
    m, n = A.shape
    if not (1 <= r <= k <= min(m, n)):
        raise ValueError("need 1 <= r <= k <= min(m, n)")
    X = (S @ A).T
    Q, R = _thin_qr(X)
    M = A @ Q
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    US = U[:, :r] * s[:r]
    QV = Q @ Vh[:r, :].T
    B = US @ QV.T
    err = float(np.linalg.norm(A - B))
    out = {"US": US, "Vt": QV.T.copy(), "sigma": s.copy(), "err": err,
           "normA2": float(np.sum(A * A)), "Q": Q, "R": R}
    if dense:
        out["B"] = B
    return out


def scw_svd_form(A, S, r: int) -> np.ndarray:
    """Algorithm 1 as printed, with the thin SVD of SA in line 1."""
    A = np.asarray(A, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    _, _, Vh = np.linalg.svd(S @ A, full_matrices=False)
    V = Vh.T
    U, s, Wh = np.linalg.svd(A @ V, full_matrices=False)
    AVr = (U[:, :r] * s[:r]) @ Wh[:r, :]
    return AVr @ V.T


def optimal_error(A, r: int) -> float:
    """||A - A_opt||_F for the best rank-r A_opt (Eckart-Young, Section 1)."""
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    return float(np.sqrt(np.sum(s[r:] ** 2)))


def test_error(errs, opt_errs) -> float:
    """Eq. 4.1: mean over the test set of (err - opt) / opt."""
    errs = np.asarray(errs, dtype=np.float64)
    opt = np.asarray(opt_errs, dtype=np.float64)
    return float(np.mean((errs - opt) / opt))


test_error.__test__ = False  # not a pytest test despite the name


def scw_batch(As, S, r: int):
    """Per-matrix SCW errors for a batch sharing one sketch S."""
    return [scw(A, S, r, dense=False)["err"] for A in As]
