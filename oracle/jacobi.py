"""Cyclic Jacobi eigen-solver for small symmetric matrices (FP64, plain loops).

TEST INFRASTRUCTURE ONLY (see ``oracle/mds.py``).  It is a second eigen
routine, independent of the LAPACK ``eigh`` that ``classical_mds`` calls, so
that brute-force classical MDS on tiny inputs (Section 2, steps 1-4) can be
checked against an eigen-solver that shares nothing with it.  Method: the
cyclic-by-row Jacobi method (Golub & Van Loan, "Matrix Computations",
Section 8.5): sweep over all (p, q) pairs, annihilate a_pq with the plane
rotation of the 2 x 2 symmetric Schur decomposition, until the off-diagonal
Frobenius norm is below tol * ||A||_F.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_eigh(A, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigenvalues (ascending) and eigenvectors (columns) of symmetric A."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    fro = math.sqrt(float(np.sum(A * A)))
    for _ in range(max_sweeps):
        off = math.sqrt(float(np.sum(np.triu(A, 1) ** 2)) * 2.0)
        if off <= tol * fro:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                # 2x2 symmetric Schur: choose (c, s) so that the rotated a_pq is 0.
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J on rows/columns p and q.
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    lam = np.diag(A).copy()
    order = np.argsort(lam)
    return lam[order], V[:, order]
