"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own arithmetic: exact recovery
of planted structure, closed forms, the paper's Proposition 1, invariants
(Eq. (1), zero row sums after double centering), brute force with a second,
independent eigen-solver, and the Table 1 correlation band.  The
``test_planted_*`` tests plant a plausible mistake in a copy of an oracle
function and show that the matching pin catches it.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_orth(r, rng, det_sign=1.0):
    Qm, R = np.linalg.qr(rng.standard_normal((r, r)))
    Qm = Qm * np.sign(np.diag(R))[None, :]
    if np.sign(np.linalg.det(Qm)) != det_sign:
        Qm[:, 0] = -Qm[:, 0]
    return Qm


def planted_rank_r(n, r, d, rng, scales=None):
    """n points whose centred cloud spans exactly r dims, embedded in R^d."""
    scales = np.linspace(6.0, 2.0, r) if scales is None else np.asarray(scales)
    Z = rng.standard_normal((n, r)) * scales
    E = np.linalg.qr(rng.standard_normal((d, r)))[0]          # d x r orthonormal
    Y = Z @ E.T + rng.standard_normal(d)[None, :] * 3.0         # plus a shift
    return Z - Z.mean(axis=0), Y


def non_euclidean_delta(n, rng, r):
    """Symmetric, zero-diagonal, non-Euclidean Delta whose top r eigenvalues of
    -1/2 P Delta P are clearly positive."""
    _, Y = planted_rank_r(n, r + 2, r + 4, rng)
    D = O.sq_dist(Y, Y)
    E = rng.uniform(0.0, 0.3, size=(n, n))
    D = D + (E + E.T)
    np.fill_diagonal(D, 0.0)
    return D


# ------------------------------------------------------------ check functions
# Each returns an error; the pins assert it is tiny, the planted tests that a
# mutated oracle function makes it large.


def err_exact_recovery(classical=O.classical_mds, n=60, r=3, seed=0):
    rng = np.random.default_rng(seed)
    Zc, Y = planted_rank_r(n, r, 7, rng)
    X, lam, _, _ = classical(O.sq_dist(Y, Y), r)
    s2 = np.linalg.svd(Zc, compute_uv=False) ** 2
    return max(O.aligned_rel_error(X, Zc), float(np.max(np.abs(lam - s2) / s2)))


def err_landmarks_reproduce(gower=O.gower_interpolate, n=40, r=3, seed=1):
    rng = np.random.default_rng(seed)
    D = non_euclidean_delta(n, rng, r)
    X1, lam, _, _ = O.classical_mds(D, r)
    Xd = gower(X1, lam, D, D)
    return float(np.max(np.abs(Xd - X1)) / np.max(np.abs(X1)))


def err_prop1(gower=O.gower_interpolate, lmds=O.lmds_triangulate, seed=2):
    rng = np.random.default_rng(seed)
    D = non_euclidean_delta(50, rng, 4)
    X1, lam, V, _ = O.classical_mds(D, 4)
    A2 = rng.uniform(0.0, 60.0, size=(17, 50))
    g = gower(X1, lam, D, A2)
    m = lmds(V, lam, D, A2)
    return float(np.max(np.abs(g - m)) / np.max(np.abs(m)))


def err_closed_form(interp=O.interpolation_mds, seed=3):
    """Gower on Euclidean data = projection of the points, centred at the
    landmark mean, on the landmarks' principal axes (right singular vectors of
    the centred landmark matrix, from an SVD rather than from Q)."""
    rng = np.random.default_rng(seed)
    n, d, l, r = 500, 9, 60, 3
    Y = rng.standard_normal((n, d)) * np.array([5.0, 4.0, 3.0] + [1.0] * (d - 3))
    idx = rng.permutation(n)[:l]
    X, var, ex = interp(Y, idx, r)
    L = Y[idx]
    ybar = L.mean(axis=0)
    _, s, Wt = np.linalg.svd(L - ybar, full_matrices=False)
    Xcf = (Y - ybar) @ Wt[:r].T
    Xcf = Xcf * np.sign(np.sum(Xcf * X, axis=0))[None, :]    # per-axis sign
    e1 = float(np.max(np.abs(X - Xcf)) / np.max(np.abs(Xcf)))
    e2 = float(np.max(np.abs(var * l - s[:r] ** 2) / s[:r] ** 2))
    return max(e1, e2)


def err_procrustes(proc=O.procrustes, det_sign=1.0, seed=4):
    rng = np.random.default_rng(seed)
    c, r = 25, 6
    B = rng.standard_normal((c, r)) * 3
    T0 = rand_orth(r, rng, det_sign)
    t0 = rng.standard_normal(r)
    A = B @ T0 + t0[None, :]
    T, t = proc(A, B)
    return max(float(np.max(np.abs(T - T0))), float(np.max(np.abs(t - t0))))


def err_dc_exact(dc=O.divide_conquer_mds, seed=5):
    rng = np.random.default_rng(seed)
    n, r = 1500, 4
    Zc, Y = planted_rank_r(n, r, 8, rng)
    part = W.partitions_uneven(n, 12, 200, 330, seed)
    X, lam_bar, _ = dc(Y, part.anchors, part.ptr, part.own, r)
    return O.aligned_rel_error(X, Zc)


# ------------------------------------------------------------------ the pins


def test_unit_square_golden():
    """Worked closed form: the corners of the unit square."""
    vals = {}
    with open(os.path.join(GOLDEN, "unit_square.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = np.array([float(x) for x in v])
    D = vals["delta"].reshape(4, 4)
    Ysq = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=float)
    assert np.array_equal(O.sq_dist(Ysq, Ysq), D)
    Q = O.double_center(D)
    lam = np.sort(np.linalg.eigvalsh(Q))[::-1]
    assert np.allclose(lam, vals["eigenvalues"], atol=1e-14)
    X, lam2, _, _ = O.classical_mds(D, 2)
    assert np.allclose(lam2, [1.0, 1.0], atol=1e-14)
    assert O.aligned_rel_error(X, Ysq - 0.5) < 1e-14


def test_sq_dist_brute_force():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((7, 5))
    B = rng.standard_normal((4, 5))
    D = O.sq_dist(A, B)
    for i in range(7):
        for j in range(4):
            s = 0.0
            for k in range(5):
                s += (A[i, k] - B[j, k]) ** 2
            assert abs(D[i, j] - s) <= 1e-14 * max(1.0, s)


def test_double_center_identities():
    """Q of a Euclidean Delta is the Gram matrix of the centred points, and Q
    has zero row and column sums (Section 2)."""
    rng = np.random.default_rng(11)
    Y = rng.standard_normal((30, 6)) * 4 + 2
    Yc = Y - Y.mean(axis=0)
    Q = O.double_center(O.sq_dist(Y, Y))
    assert np.max(np.abs(Q - Yc @ Yc.T)) < 1e-12 * np.max(np.abs(Q))
    D = non_euclidean_delta(35, rng, 3)
    Q2 = O.double_center(D)
    assert np.max(np.abs(Q2.sum(axis=0))) < 1e-12 * np.max(np.abs(Q2))
    assert np.max(np.abs(Q2.sum(axis=1))) < 1e-12 * np.max(np.abs(Q2))


@pytest.mark.parametrize("n,r,seed", [(12, 2, 0), (60, 3, 1), (200, 5, 2)])
def test_exact_recovery(n, r, seed):
    assert err_exact_recovery(n=n, r=r, seed=seed) < 1e-11


def test_eq1_variance():
    """Eq. (1): X^T X = Lambda_r and the columns of X are centred."""
    rng = np.random.default_rng(12)
    D = non_euclidean_delta(45, rng, 4)
    X, lam, _, _ = O.classical_mds(D, 4)
    assert np.max(np.abs(X.T @ X - np.diag(lam))) < 1e-10 * lam[0]
    assert np.max(np.abs(X.mean(axis=0))) < 1e-12 * np.sqrt(lam[0])


@pytest.mark.parametrize("euclid", [True, False])
def test_brute_force_jacobi(euclid):
    """Classical MDS with LAPACK eigh vs the same steps with cyclic Jacobi."""
    rng = np.random.default_rng(13)
    if euclid:
        Y = rng.standard_normal((40, 6)) * np.array([5, 4, 3, 1, 1, 1.0])
        D = O.sq_dist(Y, Y)
    else:
        D = non_euclidean_delta(40, rng, 3)
    r = 3
    X, lam, _, _ = O.classical_mds(D, r)
    Q = -0.5 * (np.eye(40) - 1 / 40) @ D @ (np.eye(40) - 1 / 40)    # matrix form of P Delta P
    lj, Vj = O.jacobi_eigh(Q)
    lj, Vj = lj[::-1][:r], Vj[:, ::-1][:, :r]
    assert np.max(np.abs(lam - lj) / lj) < 1e-12
    Xj = Vj * np.sqrt(lj)
    Xj = Xj * np.sign(np.sum(Xj * X, axis=0))
    assert np.max(np.abs(X - Xj)) < 1e-10 * np.max(np.abs(X))


def test_rank_error():
    Y = np.random.default_rng(14).standard_normal((20, 2))
    with pytest.raises(O.RankError):
        O.classical_mds(O.sq_dist(Y, Y), 3)


def test_landmarks_reproduce_themselves():
    assert err_landmarks_reproduce() < 1e-12


def test_prop1_lmds_equals_gower():
    assert err_prop1() < 1e-12


def test_closed_form_projection():
    assert err_closed_form() < 1e-10


@pytest.mark.parametrize("m", [1, 7, 60, 440])
def test_block_size_invariance(m):
    """Eq. (2) is valid for any m; blocks of 1 are the one-point-at-a-time
    scheme of RMDS."""
    rng = np.random.default_rng(15)
    Y = rng.standard_normal((500, 8)) * np.array([4, 3, 2, 1, 1, 1, 1, 1.0])
    idx = rng.permutation(500)[:60]
    Xref, _, _ = O.interpolation_mds(Y, idx, 3, m=60)
    X, _, _ = O.interpolation_mds(Y, idx, 3, m=m)
    assert np.max(np.abs(X - Xref)) < 1e-12 * np.max(np.abs(Xref))


def test_p1_reductions():
    """n <= l: interpolation MDS and divide-and-conquer MDS are classical MDS."""
    rng = np.random.default_rng(16)
    Y = rng.standard_normal((50, 5)) * np.array([4, 3, 2, 1, 1.0])
    Xc, lamc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    idx = np.arange(50)
    Xi, var, _ = O.interpolation_mds(Y, idx, 3)
    assert np.max(np.abs(Xi - Xc)) < 1e-12 * np.max(np.abs(Xc))
    assert np.allclose(var * 50, lamc, rtol=1e-14)
    Xd, lamd, _ = O.divide_conquer_mds(Y, np.arange(5), np.array([0, 45]), np.arange(5, 50), 3)
    assert O.aligned_rel_error(Xd, Xc) < 1e-12
    assert np.allclose(lamd * 50, lamc, rtol=1e-12)


@pytest.mark.parametrize("det_sign", [1.0, -1.0])
def test_procrustes_recovers_planted_map(det_sign):
    assert err_procrustes(det_sign=det_sign) < 1e-12


def test_dc_exact_recovery():
    assert err_dc_exact() < 1e-10


def err_sign_convention(sign=O.sign_convention):
    """Columns whose entry of largest magnitude is known by construction:
    col 0 has its largest |.| at row 1 (negative: flipped), col 1 at row 0
    (positive: kept), col 2 a tie of |.| = 0.5 between rows 1 (negative) and
    3 (positive) that the lowest row index decides (flipped), col 3 a tie
    between rows 0 (positive) and 2 (negative) (kept)."""
    V = np.array([[0.1, 0.9, 0.2, 0.5],
                  [-0.7, -0.3, -0.5, 0.1],
                  [0.2, 0.1, 0.1, -0.5],
                  [0.3, 0.2, 0.5, 0.0]])
    want = V * np.array([-1.0, 1.0, -1.0, 1.0])[None, :]
    return float(np.max(np.abs(sign(V) - want)))


def test_sign_convention_hand_built():
    assert err_sign_convention() == 0.0
    # the input is not modified, and a column of one sign is a fixed point
    V = -np.eye(3)
    assert np.array_equal(O.sign_convention(V), np.eye(3)) and np.array_equal(V, -np.eye(3))


def test_planted_sign_convention_signed_max():
    def bad(V):                                   # largest signed entry instead of largest |.|
        V = V.copy()
        for i in range(V.shape[1]):
            if V[int(np.argmax(V[:, i])), i] < 0:
                V[:, i] = -V[:, i]
        return V
    assert err_sign_convention(sign=bad) > 0.1

    def bad_tie(V):                               # highest index wins a tie
        V = V.copy()
        for i in range(V.shape[1]):
            a = np.abs(V[:, i])
            k = len(a) - 1 - int(np.argmax(a[::-1]))
            if V[k, i] < 0:
                V[:, i] = -V[:, i]
        return V
    assert err_sign_convention(sign=bad_tie) > 0.1


def test_dc_parts_exact_recovery():
    """A subset of the parts (the first one not included), each solved once:
    on rank-r data its aligned rows are the planted points up to one
    orthogonal map, and they equal the same rows of the whole computation."""
    rng = np.random.default_rng(6)
    n, r = 1500, 4
    Zc, Y = planted_rank_r(n, r, 8, rng)
    part = W.partitions_uneven(n, 12, 200, 330, 6)
    got = O.divide_conquer_parts(Y, part.anchors, part.ptr, part.own, [2, part.p - 1], r)
    rows = np.concatenate([g[0] for g in got])
    Xs = np.vstack([g[1] for g in got])
    assert O.aligned_rel_error(Xs, Zc[rows]) < 1e-10
    X, _, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, r)
    assert np.array_equal(X[rows], Xs)


def test_dc_part_matches_whole():
    rng = np.random.default_rng(17)
    Y = rng.standard_normal((900, 6)) * np.array([4, 3, 2, 1, 1, 1.0])
    part = W.partitions_uneven(900, 10, 150, 220, 7)
    X, _, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 3)
    for j in (0, 2):
        rows, Xj, _ = O.divide_conquer_part(Y, part.anchors, part.ptr, part.own, j, 3)
        assert np.array_equal(X[rows], Xj)


def test_embed_new_matches_interpolation():
    rng = np.random.default_rng(18)
    Y = rng.standard_normal((400, 7)) * np.array([4, 3, 2, 1, 1, 1, 1.0])
    idx = rng.permutation(400)[:50]
    X, _, ex = O.interpolation_mds(Y, idx, 3)
    model = dict(ex, L=Y[idx])
    assert np.max(np.abs(O.embed_new(model, Y) - X)) < 1e-10 * np.max(np.abs(X))


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_correlation.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, q025, mean, q975 = line.split()
            rows[k] = (float(q025), float(mean), float(q975))
    return rows


def test_table1_correlation_band():
    """Statistical band, not parity: on the paper's simulation design (k=100,
    h=r=10, l=250 for interpolation, l=400 and c=5r=50 for D&C), the aligned
    columns correlate with the dominant columns at or above Table 1's q0.025."""
    t1 = _table1()
    n, d, h = 20_000, 100, 10
    Y = W.gaussian_dominant(n, d, h, seed=21)
    idx = W.landmarks(n, 250, seed=21)
    X, _, _ = O.interpolation_mds(Y, idx, h)
    cor = O.column_correlations(X, Y[:, :h])
    assert cor.mean() >= t1["interpolation"][0]
    part = W.partitions_equal(n, 400, 50, seed=21)
    Xd, _, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, h)
    cor_d = O.column_correlations(Xd, Y[:, :h])
    assert cor_d.mean() >= t1["divide_and_conquer"][0]


# --------------------------------------------------------- planted mistakes


def test_planted_wrong_centering_sign():
    def bad(Delta, r, rank_tol=1e-12):
        Q = -O.double_center(Delta)                       # sign flipped
        lam, V = np.linalg.eigh(Q)
        o = np.argsort(lam)[::-1][:r]
        lam = np.abs(lam[o])
        return V[:, o] * np.sqrt(lam), lam, V[:, o], Q
    assert err_exact_recovery(classical=bad) > 1e-3


def test_planted_gower_dropped_q1():
    def bad(X1, lam, Delta1, A2):
        l = X1.shape[0]
        return (1.0 / (2 * l)) * (-A2) @ X1 @ np.diag(l / lam)
    assert err_landmarks_reproduce(gower=bad) > 1e-3
    assert err_prop1(gower=bad) > 1e-3


def test_planted_gower_wrong_scale():
    def bad(X1, lam, Delta1, A2):                          # S_1 with 1/(l-1)
        return O.gower_interpolate(X1, lam * X1.shape[0] / (X1.shape[0] - 1), Delta1, A2)
    assert err_landmarks_reproduce(gower=bad) > 1e-3


def test_planted_procrustes_transposed():
    def bad(A, B):
        T, t = O.procrustes(A, B)
        return T.T, A.mean(axis=0) - T @ B.mean(axis=0)
    assert err_procrustes(proc=bad) > 1e-3


def test_planted_dc_shift_sign():
    def bad_proc(A, B):
        T, t = O.procrustes(A, B)
        return T, -t
    import oracle.mds as M
    orig = M.procrustes
    M.procrustes = bad_proc
    try:
        e = err_dc_exact()
    finally:
        M.procrustes = orig
    assert e > 1e-3


def test_planted_interp_transposed_axes():
    def bad(Y, idx, r, m=None, rank_tol=1e-12):
        X, var, ex = O.interpolation_mds(Y, idx, r, m, rank_tol)
        return X[:, ::-1] * np.array([1.0, 1.0, 1.0001]), var, ex   # axes swapped / scaled
    assert err_closed_form(interp=bad) > 1e-5
