"""Plain CPU FP64 oracle for the paper's other big-data MDS variants.

TEST INFRASTRUCTURE ONLY, like ``oracle/mds.py``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it; the CUDA
product path shares no code with it.

  affine_interpolation   Eq. (2) for points given by Euclidean coordinates,
                         rewritten through the Section 2 identity
                         Q_1 = L_c L_c^T: a projection on the landmarks'
                         principal axes.
  maxmin_landmarks       LMDS's MaxMin greedy choice of the first subset
                         (Section 3.1).
  pivot_mds              pivot MDS (Section 3.1): the SVD of the n x l block
                         C of Q between all points and the pivots.
  fast_mds               fast MDS (Section 3.3): recursive division, classical
                         MDS on the leaves, Procrustes alignment of every
                         subset to an alignment configuration.

Readings of points the paper leaves open:
  * MaxMin: the first landmark is an input (the paper's implementations draw
    it at random); each next one maximises the smallest squared Euclidean
    distance to those already chosen; ties go to the lowest row index among
    the points not yet chosen.
  * Pivot MDS: C = Q[:, pivots] with Q = -1/2 P Delta P over all n points
    (the paper's definition).  With C = U Sigma W^T, the eigenvectors of Q
    are estimated by U_r and its eigenvalues by sigma_i sqrt(n / l) (for
    pivots drawn at random V_P^T V_P ~ (l/n) I, so C C^T ~ (l/n) Q^2);
    X = U_r (sigma_r sqrt(n / l))^{1/2}, with the sign convention of
    classical MDS, and the variance estimates are lambda / n (Eq. (1)).
  * Fast MDS: the random division is an input (``workloads.fast_mds_tree``:
    p = floor(l / s) subsets of ceil(m / p) points, a too-small last one
    folded into the one before); the sampling points of a subset are its
    first s points; lambda_bar averages lambda^j / n_j over the subsets on
    which classical MDS runs (the leaves).
"""
from __future__ import annotations

import numpy as np

from .mds import classical_mds, double_center, procrustes, sign_convention, sq_dist


def affine_interpolation(Y, landmark_idx, r: int, rank_tol: float = 1e-12):
    """Interpolation MDS (Section 3.1) for rows given by coordinates.

    Classical MDS of the landmarks L gives V_r, Lambda_r.  For Euclidean
    distances Q_1 = L_c L_c^T (Section 2, L_c = L - 1 y_L^T with y_L the
    landmark mean), and Eq. (2) becomes Xdot = (Y - 1 y_L^T) U_r with
    U_r = L_c^T V_r Lambda_r^{-1/2}; the landmarks get X_1 back.
    Returns (X n x r, var = lambda / l, U_r d x r)."""
    Y = np.asarray(Y, dtype=np.float64)
    idx = np.asarray(landmark_idx, dtype=np.int64)
    L = Y[idx]
    _, lam, V, _ = classical_mds(sq_dist(L, L), r, rank_tol)
    y_L = L.mean(axis=0)
    U = (L - y_L).T @ V @ np.diag(lam ** -0.5)
    return (Y - y_L) @ U, lam / len(idx), U


def maxmin_landmarks(Y, l: int, first: int) -> np.ndarray:
    """LMDS's MaxMin choice of l landmarks (Section 3.1), starting from row
    ``first``: each next landmark is the row whose smallest squared distance
    to the landmarks chosen so far is largest.  Returns the l row indices in
    the order chosen."""
    Y = np.asarray(Y, dtype=np.float64)
    n = Y.shape[0]
    if not 0 < l <= n or not 0 <= first < n:
        raise ValueError("need 0 < l <= n and 0 <= first < n")
    chosen = [int(first)]
    taken = np.zeros(n, dtype=bool)
    taken[first] = True
    mind = sq_dist(Y, Y[[first]])[:, 0]
    for _ in range(1, l):
        score = np.where(taken, -1.0, mind)
        nxt = int(np.argmax(score))          # lowest index on ties
        chosen.append(nxt)
        taken[nxt] = True
        mind = np.minimum(mind, sq_dist(Y, Y[[nxt]])[:, 0])
    return np.asarray(chosen, dtype=np.int64)


def pivot_mds(Y, pivot_idx, r: int):
    """Pivot MDS (Section 3.1): C is the n x l block of Q = -1/2 P Delta P
    (all n points) between every point and the pivots; the SVD C = U Sigma W^T
    approximates the eigendecomposition of Q (eigenvectors U_r, eigenvalues
    sigma_i sqrt(n / l)), and X = U_r diag(sigma_r sqrt(n / l))^{1/2}.
    Returns (X n x r, var = lambda / n, lambda r)."""
    Y = np.asarray(Y, dtype=np.float64)
    piv = np.asarray(pivot_idx, dtype=np.int64)
    n, l = Y.shape[0], len(piv)
    Q = double_center(sq_dist(Y, Y))
    C = Q[:, piv]
    U, sig, _ = np.linalg.svd(C, full_matrices=False)
    lam = sig[:r] * np.sqrt(n / l)
    V = sign_convention(U[:, :r])
    return V * np.sqrt(lam)[None, :], lam / n, lam


def fast_mds(Y, tree, r: int, s: int, rank_tol: float = 1e-12):
    """Fast MDS (Section 3.3) over the random division ``tree``
    (``workloads.FastNode``).

    A leaf's configuration is its classical MDS.  At an inner node with
    subsets j = 1..p: the first s points of every subset form the alignment
    set, whose classical MDS is X_align; each subset's configuration X_j is
    aligned by Procrustes on its sampling points,
    X_align,j^s ~ X_j^s T_j + 1 t_j^T, giving X_j T_j + 1 t_j^T; the aligned
    subsets, concatenated, are the node's configuration.  The root's
    configuration is returned in original row order, with lambda_bar =
    mean over the leaves of lambda^j / n_j.  Returns (X n x r, lambda_bar r,
    extras with the per-leaf (rows, lambda))."""
    Y = np.asarray(Y, dtype=np.float64)
    leaves = []

    def solve(node):
        if not node.children:
            Yn = Y[node.idx]
            X, lam, _, _ = classical_mds(sq_dist(Yn, Yn), r, rank_tol)
            leaves.append((node.idx, lam))
            return X
        parts = [solve(ch) for ch in node.children]
        align_rows = np.concatenate([ch.idx[:s] for ch in node.children])
        Ya = Y[align_rows]
        X_align, _, _, _ = classical_mds(sq_dist(Ya, Ya), r, rank_tol)
        out = []
        for j, Xj in enumerate(parts):
            T, t = procrustes(X_align[j * s:(j + 1) * s], Xj[:s])
            out.append(Xj @ T + t[None, :])
        return np.vstack(out)

    Xroot = solve(tree)
    X = np.empty_like(Xroot)
    X[tree.idx] = Xroot
    lam_bar = np.mean([lam / len(rows) for rows, lam in leaves], axis=0)
    return X, lam_bar, {"leaves": leaves}
