"""Oracle: LAPACK-free PSD projection by the cyclic Jacobi method (TEST INFRASTRUCTURE).

Pi(X) = Q max(0, W) Q^T (Sec. 4, parallel PSD cone projection) with the
eigendecomposition X = Q W Q^T computed by the classical cyclic-by-row
Jacobi method of Golub & Van Loan (Matrix Computations, Sec. 8.5): sweep over
the pairs (p, q), p < q, in row order; each pair is annihilated by the
2 x 2 symmetric Schur rotation (c, s) with
    tau = (a_qq - a_pp) / (2 a_pq),   t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
    c = 1 / sqrt(1 + t^2),            s = t c   (sign(0) = +1),
applied as A <- J^T A J and V <- V J, J the identity except
J[p, p] = J[q, q] = c, J[p, q] = s, J[q, p] = -s. Sweeps stop when
off(A) <= tol ||A||_F (off = Frobenius norm of the off-diagonal part), at most
max_sweeps. Plain FP64 NumPy, one rotation at a time, no blocking and no
reordering: slow, and meant to be read against the method. It shares nothing
with the CUDA eigensolvers of the library, which use a parallel (round-robin)
ordering.
"""
from __future__ import annotations

import numpy as np

TOL = 1e-14
MAX_SWEEPS = 60


def sym_schur2(A: np.ndarray, p: int, q: int):
    """(c, s) of the rotation that zeroes A[p, q] of the symmetric 2 x 2 block."""
    apq = A[p, q]
    if apq == 0.0:
        return 1.0, 0.0
    tau = (A[q, q] - A[p, p]) / (2.0 * apq)
    t = (1.0 if tau >= 0.0 else -1.0) / (abs(tau) + np.sqrt(1.0 + tau * tau))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, t * c


def off(A: np.ndarray) -> float:
    """Frobenius norm of the off-diagonal part, summed over the off-diagonal
    entries themselves (||A||_F^2 - sum a_ii^2 would cancel near convergence)."""
    mask = ~np.eye(A.shape[0], dtype=bool)
    return float(np.sqrt(np.sum(A[mask] ** 2)))


def eig_jacobi(X: np.ndarray, tol: float = TOL, max_sweeps: int = MAX_SWEEPS):
    """(eigenvalues, eigenvectors as columns, sweeps used) of the symmetric X."""
    A = 0.5 * (np.asarray(X, dtype=np.float64) + np.asarray(X, dtype=np.float64).T)
    n = A.shape[0]
    V = np.eye(n)
    fro = float(np.linalg.norm(A))
    sweeps = 0
    while sweeps < max_sweeps and off(A) > tol * fro:
        for p in range(n - 1):
            for q in range(p + 1, n):
                c, s = sym_schur2(A, p, q)
                if s == 0.0:
                    continue
                # A <- J^T A J: rotate columns p, q, then rows p, q
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * ap - s * aq, s * ap + c * aq
                ap, aq = A[p, :].copy(), A[q, :].copy()
                A[p, :], A[q, :] = c * ap - s * aq, s * ap + c * aq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
        sweeps += 1
    return np.diag(A).copy(), V, sweeps


def project_block(X: np.ndarray, tol: float = TOL, max_sweeps: int = MAX_SWEEPS) -> np.ndarray:
    """Pi_{S+}(X) = Q max(0, W) Q^T with (W, Q) from the cyclic Jacobi method."""
    w, Q, _ = eig_jacobi(X, tol, max_sweeps)
    return (Q * np.maximum(w, 0.0)) @ Q.T
