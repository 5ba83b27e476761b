"""Plain CPU FP64 oracle for classical, interpolation and divide-and-conquer MDS.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or call this module.  The CUDA product path never does; it shares no code
with this file.

Every function restates one passage of Delicado & Pachon-Garcia,
"Multidimensional scaling for big data" (arXiv 2007.11919), in the paper's
notation and order of steps, with no blocking, fusion or reordering beyond
what that passage states.  Library primitives used as single steps:
``numpy.linalg.eigh`` (the symmetric eigendecomposition of Section 2 step 2),
``numpy.linalg.svd`` (the SVD inside orthogonal Procrustes) and matrix
products.

Readings of points the paper leaves open:
  * Delta holds squared Euclidean distances (Section 2); they are formed
    here in the direct difference form sum_k (y_ik - y_jk)^2, never through
    norms, so this side has no cancellation to guard against.
  * "the r greatest non-negative eigenvalues" (Section 2, step 3): fewer
    than r eigenvalues above ``rank_tol * lambda_1`` raises ``RankError``.
  * Eigenvector sign: each column of V is flipped so that its entry of
    largest magnitude is positive (the lowest row index wins a tie).
  * Procrustes (Section 3.2): T orthogonal, reflections allowed, no
    dilation; A ~ B T + 1 t^T solved through the SVD of B_c^T A_c.
  * Divide-and-conquer: part j is the c connecting points followed by its
    own points; X_1 is kept whole; the output is in original row order.
"""
from __future__ import annotations

import numpy as np


class RankError(ValueError):
    """Fewer than r positive eigenvalues: Lambda_r^{-1/2} is undefined."""


# ----------------------------------------------------------------- Section 2


def sq_dist(A, B, chunk_elems: int = 1 << 24) -> np.ndarray:
    """Squared Euclidean distances d^2_ij = sum_k (a_ik - b_jk)^2 (Section 2).

    Direct difference form in FP64.  ``A`` is m x k, ``B`` is l x k.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, k = A.shape
    l = B.shape[0]
    out = np.empty((m, l), dtype=np.float64)
    rows = max(1, chunk_elems // max(1, l * k))
    for i in range(0, m, rows):
        diff = A[i:i + rows, None, :] - B[None, :, :]
        out[i:i + rows] = np.einsum("ijk,ijk->ij", diff, diff)
    return out


def double_center(Delta) -> np.ndarray:
    """Q = -1/2 P Delta P written entrywise (Section 2):
    q_ij = -(d2_ij - d2_i. - d2_.j + d2_..) / 2, with the row, column and
    grand means of Delta."""
    D = np.asarray(Delta, dtype=np.float64)
    row = D.mean(axis=1)          # d2_i.
    col = D.mean(axis=0)          # d2_.j
    grand = D.mean()              # d2_..
    return -0.5 * (D - row[:, None] - col[None, :] + grand)


def sign_convention(V: np.ndarray) -> np.ndarray:
    """Flip each column so its largest-magnitude entry is positive."""
    V = V.copy()
    for i in range(V.shape[1]):
        k = int(np.argmax(np.abs(V[:, i])))
        if V[k, i] < 0:
            V[:, i] = -V[:, i]
    return V


def classical_mds(Delta, r: int, rank_tol: float = 1e-12):
    """Classical MDS of a squared-distance matrix (Section 2, steps 1-4).

    1. Q = -1/2 P Delta P.
    2. Eigen-pairs of Q sorted by decreasing eigenvalue.
    3. Keep the r largest; they must be positive.
    4. X = V_r Lambda_r^{1/2}.

    Returns (X n x r, lambda r, V n x r, Q n x n).
    """
    Q = double_center(Delta)
    lam, V = np.linalg.eigh(Q)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    lam_r, V_r = lam[:r].copy(), V[:, :r]
    if r > len(lam) or not lam_r[-1] > rank_tol * max(lam_r[0], 0.0) or lam_r[-1] <= 0:
        raise RankError(f"fewer than {r} positive eigenvalues")
    V_r = sign_convention(V_r)
    X = V_r * np.sqrt(lam_r)[None, :]
    return X, lam_r, V_r, Q


# ------------------------------------------------------- Section 3.1, Eq. (2)


def gower_interpolate(X1, lam, Delta1, A2) -> np.ndarray:
    """Gower's interpolation formula, Eq. (2), literally:
    Xdot_2 = 1/(2l) (1_m q_1^T - A^2_21) X_1 S_1^{-1},
    q_1 = diag(Q_1), Q_1 = -1/2 P Delta_1 P, S_1 = Lambda_1 / l (Eq. (1)).
    ``A2`` is the m x l matrix of squared distances to the l first points."""
    X1 = np.asarray(X1, dtype=np.float64)
    A2 = np.asarray(A2, dtype=np.float64)
    l = X1.shape[0]
    m = A2.shape[0]
    Q1 = double_center(Delta1)
    q1 = np.diag(Q1)
    S1 = np.diag(np.asarray(lam, dtype=np.float64)) / l
    ones_m = np.ones((m, 1))
    return (1.0 / (2.0 * l)) * (ones_m @ q1[None, :] - A2) @ X1 @ np.linalg.inv(S1)


def lmds_triangulate(V1, lam, Delta1, A2) -> np.ndarray:
    """Landmark-MDS distance-based triangulation, Eq. (3):
    X_2 = 1/2 (1_m d_1^T - A^2_21) V_1,r Lambda_1,r^{-1/2}, with
    d_1 = Delta_1 1_l / l the mean squared distance of each landmark."""
    V1 = np.asarray(V1, dtype=np.float64)
    A2 = np.asarray(A2, dtype=np.float64)
    D1 = np.asarray(Delta1, dtype=np.float64)
    l = D1.shape[0]
    m = A2.shape[0]
    d1 = D1 @ np.ones(l) / l
    return 0.5 * (np.ones((m, 1)) @ d1[None, :] - A2) @ V1 @ np.diag(np.asarray(lam) ** -0.5)


def interpolation_mds(Y, landmark_idx, r: int, m: int | None = None, rank_tol: float = 1e-12):
    """Interpolation MDS (Section 3.1).

    The first subset is the l points ``landmark_idx`` (drawn at random by the
    caller); classical MDS gives X_1; the other points, taken in increasing
    row order, are interpolated with Eq. (2) in blocks of m (default m = l);
    the pieces are put back in original row order.  Returns (X n x r,
    var = lambda / l, extras dict with X1, lam, V, Delta1)."""
    Y = np.asarray(Y)
    n = Y.shape[0]
    idx = np.asarray(landmark_idx, dtype=np.int64)
    l = len(idx)
    if m is None:
        m = l
    L = Y[idx].astype(np.float64)
    Delta1 = sq_dist(L, L)
    X1, lam, V1, _ = classical_mds(Delta1, r, rank_tol)
    X = np.empty((n, r), dtype=np.float64)
    X[idx] = X1
    is_lm = np.zeros(n, dtype=bool)
    is_lm[idx] = True
    rest = np.nonzero(~is_lm)[0]
    for b in range(0, len(rest), m):
        blk = rest[b:b + m]
        A2 = sq_dist(Y[blk].astype(np.float64), L)
        X[blk] = gower_interpolate(X1, lam, Delta1, A2)
    return X, lam / l, {"X1": X1, "lam": lam, "V": V1, "Delta1": Delta1}


def embed_new(model: dict, Ynew) -> np.ndarray:
    """Eq. (2) applied to new points against a stored first subset
    (``model`` as returned in the extras of ``interpolation_mds`` plus the
    landmark rows under key "L")."""
    A2 = sq_dist(np.asarray(Ynew, dtype=np.float64), model["L"])
    return gower_interpolate(model["X1"], model["lam"], model["Delta1"], A2)


# --------------------------------------------------------------- Section 3.2


def procrustes(A, B):
    """Orthogonal Procrustes with translation (Section 3.2): T (r x r,
    orthogonal, reflections allowed, no dilation) and t (r) such that
    A ~ B T + 1 t^T in least squares.  Centre both, C = B_c^T A_c = U S W^T,
    T = U W^T, t = a_bar - T^T b_bar."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    a_bar = A.mean(axis=0)
    b_bar = B.mean(axis=0)
    C = (B - b_bar).T @ (A - a_bar)
    U, _, Wt = np.linalg.svd(C)
    T = U @ Wt
    t = a_bar - T.T @ b_bar
    return T, t


def _part_classical(job):
    """Classical MDS of one part from its rows (Section 3.2: each part is an
    ordinary classical-MDS problem).  ``job`` = (rows of the part, r,
    rank_tol); returns (X_j, lambda^j)."""
    Yj, r, rank_tol = job
    Yj = np.asarray(Yj, dtype=np.float64)
    Xj, lam_j, _, _ = classical_mds(sq_dist(Yj, Yj), r, rank_tol)
    return Xj, lam_j


def _members(anchors, ptr, own, j):
    """Points of part j: the c connecting points, then its own points."""
    return np.concatenate([anchors, np.asarray(own[ptr[j]:ptr[j + 1]], dtype=np.int64)])


def divide_conquer_mds(Y, anchors, ptr, own, r: int, rank_tol: float = 1e-12, map_fn=map):
    """Divide-and-conquer MDS (Section 3.2).

    Part j's points are the c connecting points ``anchors`` followed by its
    own points ``own[ptr[j]:ptr[j+1]]``.  Classical MDS on each part gives
    X_j and lambda^j; each X_j (j >= 2) is aligned to X_1 by Procrustes on
    the connecting points, X_1^c ~ X_j^c T_j + 1 t_j^T; the aligned rows
    without the connecting points, X_j^a T_j + 1 t_j^T, and X_1 whole are put
    in original row order.  lambda_bar_i = (1/p) sum_j lambda_i^j / n_j.
    The parts' classical MDS problems are independent of one another
    (Section 3.2 solves them separately); ``map_fn`` (default: the builtin
    map, in part order) may run them in parallel processes.
    Returns (X n x r, lambda_bar r, extras)."""
    Y = np.asarray(Y)
    anchors = np.asarray(anchors, dtype=np.int64)
    ptr = np.asarray(ptr, dtype=np.int64)
    own = np.asarray(own, dtype=np.int64)
    c = len(anchors)
    p = len(ptr) - 1
    n = Y.shape[0]
    X = np.full((n, r), np.nan)
    lam_sum = np.zeros(r)
    members = [_members(anchors, ptr, own, j) for j in range(p)]
    solved = list(map_fn(_part_classical, [(Y[m], r, rank_tol) for m in members]))
    X1c = None
    per_part = []
    for j in range(p):
        Xj, lam_j = solved[j]
        lam_sum += lam_j / len(members[j])
        if j == 0:
            X1c = Xj[:c]
            X[members[j]] = Xj
            per_part.append((np.eye(r), np.zeros(r), lam_j))
        else:
            T, t = procrustes(X1c, Xj[:c])
            X[members[j][c:]] = Xj[c:] @ T + t[None, :]
            per_part.append((T, t, lam_j))
    return X, lam_sum / p, {"parts": per_part}


def divide_conquer_parts(Y, anchors, ptr, own, parts, r: int, rank_tol: float = 1e-12, map_fn=map):
    """The rows of the listed parts of ``divide_conquer_mds``, computed alone:
    classical MDS of part 1 (index 0, solved once whether listed or not) and
    of every listed part, each listed part j >= 2 aligned to part 1 by
    Procrustes on the connecting points (Section 3.2).  Returns a list of
    (row indices, aligned coordinates, lambda^j), one per listed part, in
    the order listed."""
    anchors = np.asarray(anchors, dtype=np.int64)
    c = len(anchors)
    parts = [int(j) for j in parts]
    need = [0] + [j for j in parts if j != 0]
    members = {j: _members(anchors, ptr, own, j) for j in need}
    solved = dict(zip(need, map_fn(_part_classical, [(np.asarray(Y)[members[j]], r, rank_tol) for j in need])))
    X1, _ = solved[0]
    out = []
    for j in parts:
        Xj, lam_j = solved[j]
        if j == 0:
            out.append((members[0], Xj, lam_j))
        else:
            T, t = procrustes(X1[:c], Xj[:c])
            out.append((members[j][c:], Xj[c:] @ T + t[None, :], lam_j))
    return out


def divide_conquer_part(Y, anchors, ptr, own, j: int, r: int, rank_tol: float = 1e-12):
    """Rows of part j of ``divide_conquer_mds``, computed alone (parts 1 and
    j, then their Procrustes alignment).  Returns (row indices, aligned
    coordinates, lambda^j)."""
    return divide_conquer_parts(Y, anchors, ptr, own, [j], r, rank_tol)[0]
