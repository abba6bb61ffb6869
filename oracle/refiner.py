"""IVY loss (Eq. 2.1) of a dense sketch and its gradient, float64.

TEST INFRASTRUCTURE: used to check the learned sketch refiner
S_theta = S_tensor + dS.

Loss.  Eq. 2.1 sums ||A - SCW(A, S, r)||_F^2 over the training set.  The
paper leaves the scale open (its baselines normalise the training matrices,
Section 4), so the refiner uses the per-sample normalised loss averaged over
a batch:

    L(S) = mean_A ||A - SCW(A, S, r)||_F^2 / ||A||_F^2.

Gradient (derived here; the paper gives none).  With X = (SA)^T = Q R,
M = A Q = U Sigma V^T and Z = U_r Sigma_r = A Q V_r, the projection identity
used in the proof of Theorem 1 (Eq. A.3) gives
||A - SCW||^2 = ||A||^2 - f with f = sum_{i<=r} sigma_i(AQ)^2.  f depends on
X only through span(X).  Differentiating the generalised eigenvalues of the
pencil (X^T A^T A X, X^T X) gives

    df/dX = 2 (A^T Z - Q V_r Sigma_r^2) W^T,   W = R^{-1} V_r  (k x r),

and since X = A^T S^T,

    df/dS = (A df/dX)^T = 2 W (A A^T Z - Z Sigma_r^2)^T        (k x m).

So dL/dS = -(2 / ||A||^2) W (A A^T Z - Z Sigma_r^2)^T per sample.  The
formula needs sigma_r(AQ) > sigma_{r+1}(AQ); the tests compare it with
central finite differences.
"""
from __future__ import annotations

import numpy as np


def scw_forward_parts(A, S, r: int):
    """Pieces of the SCW forward pass that the gradient reuses."""
    A = np.asarray(A, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    X = (S @ A).T
    Q, R = np.linalg.qr(X, mode="reduced")
    M = A @ Q
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    Vr = Vh[:r, :].T
    Z = U[:, :r] * s[:r]
    W = np.linalg.solve(R, Vr)
    normA2 = float(np.sum(A * A))
    f = float(np.sum(s[:r] ** 2))
    return {"X": X, "Q": Q, "R": R, "sigma": s, "Vr": Vr, "Z": Z, "W": W,
            "normA2": normA2, "f": f}


def _sample_loss(A, S, r):
    A = np.asarray(A, dtype=np.float64)
    X = (np.asarray(S, dtype=np.float64) @ A).T
    Q, _ = np.linalg.qr(X, mode="reduced")
    U, s, Vh = np.linalg.svd(A @ Q, full_matrices=False)
    B = (U[:, :r] * s[:r]) @ (Q @ Vh[:r, :].T).T
    return float(np.sum((A - B) ** 2) / np.sum(A * A))


def ivy_loss(S, As, r: int) -> float:
    """L(S) = mean over As of ||A - SCW(A, S, r)||_F^2 / ||A||_F^2."""
    return float(np.mean([_sample_loss(A, S, r) for A in As]))


def ivy_grad(S, As, r: int) -> np.ndarray:
    """Analytic dL/dS (k x m) of ivy_loss, averaged over the batch."""
    S = np.asarray(S, dtype=np.float64)
    g = np.zeros_like(S)
    for A in As:
        A = np.asarray(A, dtype=np.float64)
        p = scw_forward_parts(A, S, r)
        Z, W, s = p["Z"], p["W"], p["sigma"]
        T = A @ (A.T @ Z) - Z * (s[:r] ** 2)
        g += -(2.0 / p["normA2"]) * (W @ T.T)
    return g / len(As)
