"""Two-sided variant, float64 (test infrastructure).

Algorithm 3 (two-sided SCW): Q from the QR of A^T S^T, P from the QR of
A W^T, [P^T A Q]_r the truncated SVD of the l x k core, and
A_hat = P [P^T A Q]_r Q^T.

Algorithm 5 (HOOI) for the Tucker2 problem (Eq. 3.6): only modes 1 and 2 of
calA (m x n x D') are compressed, so the mode-3 factor stays the identity.
Readings of the garbled listing: the iteration counter advances once per
sweep over the modes (not inside the mode loop), the starting guess is the
HOSVD one (leading eigenvectors of the mode-1 and mode-2 Gram matrices), and
"convergent" means that ||calG||_F^2 changed by less than 1e-12 ||calA||_F^2
over a sweep, or 50 sweeps were made.
"""
from __future__ import annotations

import numpy as np

from .tensor_sketch import gram_mode1, gram_mode2, leading_eigvecs


def two_sided_scw(A, S, W, r: int):
    """Algorithm 3.  Returns dict(err, B, core_sigma)."""
    A = np.asarray(A, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    Q, _ = np.linalg.qr(A.T @ S.T, mode="reduced")
    P, _ = np.linalg.qr(A @ W.T, mode="reduced")
    core = P.T @ A @ Q
    U, s, Vh = np.linalg.svd(core, full_matrices=False)
    core_r = (U[:, :r] * s[:r]) @ Vh[:r, :]
    B = P @ core_r @ Q.T
    return {"err": float(np.linalg.norm(A - B)), "B": B, "core_sigma": s}


def hooi(As, k: int, l: int, max_sweeps: int = 50, tol: float = 1e-12):
    """Tucker2 of the training tensor by HOOI; returns (S, W, sweeps)."""
    As = [np.asarray(A, dtype=np.float64) for A in As]
    total = sum(float(np.sum(A * A)) for A in As)
    S, _ = leading_eigvecs(gram_mode1(As), k)
    W, _ = leading_eigvecs(gram_mode2(As), l)
    prev = None
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        # mode 1: project mode 2 on W, keep the top-k left singular vectors
        G1 = sum((A @ W.T) @ (A @ W.T).T for A in As)
        S, _ = leading_eigvecs(G1, k)
        # mode 2: project mode 1 on the new S
        G2 = sum((S @ A).T @ (S @ A) for A in As)
        W, _ = leading_eigvecs(G2, l)
        core = sum(float(np.sum((S @ A @ W.T) ** 2)) for A in As)
        if prev is not None and abs(core - prev) < tol * total:
            break
        prev = core
    return S, W, sweeps
