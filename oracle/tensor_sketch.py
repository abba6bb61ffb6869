"""Training side of the tensor-based method, in float64 (test infrastructure).

Section 3.1: stacking the training matrices A_1..A_D' into the tensor
calA (m x n x D') and unfolding along mode 1 gives A_(1) = [A_1 | ... | A_D']
(m x nD').  Problem (3.1) is equivalent to maximising ||S A_(1)||_F^2 over
row-orthonormal S (Eq. 3.2), i.e. the Tucker1 problem (3.3), whose solution
is S* = (U^(1))_k^T, the first k left singular vectors of A_(1).

The left singular vectors of A_(1) are the eigenvectors of
A_(1) A_(1)^T = sum_d A_d A_d^T, so the oracle forms that Gram matrix and
takes its leading eigenvectors.  The column order of the unfolding does not
change the Gram matrix, which is why the garbled column-index formula of the
tensor-basics paragraph (Section 2) does not matter here.
"""
from __future__ import annotations

import numpy as np


def gram_mode1(As) -> np.ndarray:
    """G = A_(1) A_(1)^T = sum_d A_d A_d^T  (m x m), Section 3.1 / Eq. 3.2."""
    As = [np.asarray(A, dtype=np.float64) for A in As]
    m = As[0].shape[0]
    G = np.zeros((m, m))
    for A in As:
        G += A @ A.T
    return G


def gram_mode2(As) -> np.ndarray:
    """G2 = A_(2) A_(2)^T = sum_d A_d^T A_d  (n x n).

    The mode-2 unfolding stacks the transposed slices, so its Gram matrix is
    the sum of A_d^T A_d; its leading eigenvectors give the second sketch W
    of the two-sided problem (Eq. 3.6) at the HOSVD starting point.
    """
    As = [np.asarray(A, dtype=np.float64) for A in As]
    n = As[0].shape[1]
    G = np.zeros((n, n))
    for A in As:
        G += A.T @ A
    return G


def canonical_signs(V: np.ndarray) -> np.ndarray:
    """Flip each column so its largest-magnitude entry is positive.

    Eigenvectors are defined up to sign; the paper does not fix one.  The
    entry of largest magnitude (lowest index on a tie) is made positive.
    """
    V = np.array(V, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return V


def leading_eigvecs(G: np.ndarray, k: int):
    """Top-k eigenvectors of the symmetric G as the rows of S (k x m).

    Returns (S, lam) with lam all eigenvalues in descending order.
    This is S* = (U^(1))_k^T of Section 3.1.
    """
    G = np.asarray(G, dtype=np.float64)
    lam, V = np.linalg.eigh(0.5 * (G + G.T))
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    V = canonical_signs(V[:, order[:k]])
    return V.T.copy(), lam


def train_sketch(As, k: int, l: int = 0):
    """Algorithm 2, lines 1-2: tensorise, Tucker1 along mode 1 -> S (k x m).

    With l > 0 the second sketch W (l x n) is taken from the mode-2 Gram,
    the HOSVD starting point of the Tucker2 problem (Eq. 3.6).
    Returns (S, W or None, lam1, lam2 or None).
    """
    S, lam1 = leading_eigvecs(gram_mode1(As), k)
    if l > 0:
        W, lam2 = leading_eigvecs(gram_mode2(As), l)
        return S, W, lam1, lam2
    return S, None, lam1, None
