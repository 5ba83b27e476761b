"""Pins of the oracle's big-data MDS variants (oracle/variants.py) against
what the paper and the mathematics fix: closed forms, a hand-derived MaxMin
order, the k-center 2-approximation of farthest-first choice (brute force),
special cases that reduce to classical MDS, exact recovery of planted
structure, and invariants of orthogonal alignment.  The ``test_planted_*``
tests plant a plausible mistake in a copy of a function and show that the
matching pin catches it."""
import itertools

import numpy as np
import pytest

import oracle as O
import oracle.variants as V
import workloads as W


def planted_rank_r(n, r, d, rng):
    Z = rng.standard_normal((n, r)) * np.linspace(6.0, 2.0, r)
    E = np.linalg.qr(rng.standard_normal((d, r)))[0]
    Y = Z @ E.T + rng.standard_normal(d)[None, :] * 3.0
    return Z - Z.mean(axis=0), Y


# ----------------------------------------------------- affine interpolation


def err_affine(affine=V.affine_interpolation, seed=0):
    rng = np.random.default_rng(seed)
    n, d, l, r = 400, 8, 50, 3
    Y = rng.standard_normal((n, d)) * np.array([5.0, 4.0, 3.0] + [1.0] * (d - 3)) + 2.0
    idx = rng.permutation(n)[:l]
    Xa, va, _ = affine(Y, idx, r)
    Xg, vg, ex = O.interpolation_mds(Y, idx, r)          # Eq. (2) on distances
    e1 = float(np.max(np.abs(Xa - Xg)) / np.max(np.abs(Xg)))
    e2 = float(np.max(np.abs(Xa[idx] - ex["X1"])) / np.max(np.abs(ex["X1"])))
    return max(e1, e2, float(np.max(np.abs(va - vg) / vg)))


def test_affine_equals_gower_on_coordinates():
    assert err_affine() < 1e-10


def test_planted_affine_global_mean():
    def bad(Y, idx, r, rank_tol=1e-12):            # centred at the mean of all rows
        Y = np.asarray(Y, dtype=np.float64)
        L = Y[idx]
        _, lam, Vr, _ = O.classical_mds(O.sq_dist(L, L), r)
        U = (L - L.mean(axis=0)).T @ Vr @ np.diag(lam ** -0.5)
        return (Y - Y.mean(axis=0)) @ U, lam / len(idx), U
    assert err_affine(affine=bad) > 1e-3


# --------------------------------------------------------- MaxMin landmarks


def test_maxmin_line_order():
    """x = 0, 1, 3, 7, 15 (stored shuffled).  From 0: 15 is farthest; then 7
    (gaps 1, 3, 7 to the set {0, 15}: min(7, 8) = 7 is largest); then 3
    (min(3, 4) beats 1); then 1.  From 7: 15 (8 beats 7), then 0 (7 beats
    6 and 4), then 3 (3 beats 1), then 1."""
    x = np.array([7.0, 1.0, 15.0, 0.0, 3.0])
    Y = x[:, None]
    pos = {v: i for i, v in enumerate(x)}
    got = [x[i] for i in V.maxmin_landmarks(Y, 5, pos[0.0])]
    assert got == [0.0, 15.0, 7.0, 3.0, 1.0]
    got = [x[i] for i in V.maxmin_landmarks(Y, 5, pos[7.0])]
    assert got == [7.0, 15.0, 0.0, 3.0, 1.0]


def test_maxmin_tie_lowest_index():
    """Unit-square corners (rows 1-4) around their centre (row 0).  From the
    centre the four corners tie at 1/2 (row 1 wins), then every corner left
    is 1/2 from the centre, nearer than to row 1, so rows 2-4 tie (row 2
    wins).  From corner (1,1): (0,0) is strictly farthest (2), then (0,1)
    and (1,0) tie at 1 above the centre's 1/2 (row 2 wins)."""
    Y = np.array([[0.5, 0.5], [1, 1], [0, 1], [0, 0], [1, 0]], dtype=np.float64)
    assert list(V.maxmin_landmarks(Y, 3, 0)) == [0, 1, 2]
    assert list(V.maxmin_landmarks(Y, 3, 1)) == [1, 3, 2]


def test_maxmin_invariants_and_two_approximation():
    rng = np.random.default_rng(1)
    for trial in range(20):
        n, l = 9, 3
        Y = rng.standard_normal((n, 2))
        first = int(rng.integers(n))
        S = V.maxmin_landmarks(Y, l, first)
        assert len(set(S.tolist())) == l and S[0] == first
        D = np.sqrt(O.sq_dist(Y, Y))
        # the gap of each new pick to the set before it never grows
        gaps = [D[S[k], S[:k]].min() for k in range(1, l)]
        assert all(a >= b - 1e-12 for a, b in zip(gaps, gaps[1:]))
        # covering radius within 2x of the optimal l-center (brute force)
        radius = D[:, S].min(axis=1).max()
        best = min(D[:, list(c)].min(axis=1).max() for c in itertools.combinations(range(n), l))
        assert radius <= 2.0 * best + 1e-12


def test_maxmin_duplicates_picked_once():
    Y = np.array([[0.0], [0.0], [5.0], [5.0]])
    S = V.maxmin_landmarks(Y, 4, 0)
    assert sorted(S.tolist()) == [0, 1, 2, 3]


def test_planted_maxmin_last_pick_only():
    def bad(Y, l, first):                           # distance to the newest pick only
        Y = np.asarray(Y, dtype=np.float64)
        chosen = [first]
        for _ in range(1, l):
            d = O.sq_dist(Y, Y[[chosen[-1]]])[:, 0]
            d[chosen] = -1.0
            chosen.append(int(np.argmax(d)))
        return np.asarray(chosen)
    x = np.array([7.0, 1.0, 15.0, 0.0, 3.0])
    got = [x[i] for i in bad(x[:, None], 5, 3)]
    assert got != [0.0, 15.0, 7.0, 3.0, 1.0]


# ---------------------------------------------------------------- pivot MDS


def test_pivot_all_points_is_classical():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((80, 6)) * np.array([5, 4, 3, 1, 1, 1.0])
    X, var, lam = V.pivot_mds(Y, np.arange(80), 3)
    Xc, lc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    assert np.max(np.abs(lam - lc) / lc) < 1e-10
    assert np.max(np.abs(X - Xc)) < 1e-9 * np.max(np.abs(Xc))
    assert np.allclose(var, lc / 80, rtol=1e-10)


def err_pivot_two_copies(pivot=V.pivot_mds, seed=3):
    """Two copies of a cloud, pivots = the first copy: the pivot rows of Q's
    eigenvectors satisfy V_P^T V_P = I / 2 = (l / n) I exactly, so the SVD of
    C gives Q's eigenvectors and sigma_i sqrt(n / l) its eigenvalues."""
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((60, 5)) * np.array([6, 4, 3, 2, 1.0])
    Y = np.vstack([Z, Z])
    X, _, lam = pivot(Y, np.arange(60), 3)
    Xc, lc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    return max(float(np.max(np.abs(lam - lc) / lc)), O.aligned_rel_error(X, Xc))


def test_pivot_two_copies_exact():
    assert err_pivot_two_copies() < 1e-10


def test_planted_pivot_no_rescale():
    def bad(Y, piv, r):                             # eigenvalues taken as sigma_i
        Y = np.asarray(Y, dtype=np.float64)
        C = O.double_center(O.sq_dist(Y, Y))[:, piv]
        U, sig, _ = np.linalg.svd(C, full_matrices=False)
        return O.sign_convention(U[:, :r]) * np.sqrt(sig[:r]), sig[:r] / len(Y), sig[:r]
    assert err_pivot_two_copies(pivot=bad) > 1e-3


# ----------------------------------------------------------------- fast MDS


def test_fast_small_is_classical():
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((90, 5)) * np.array([5, 3, 2, 1, 1.0])
    tree = W.fast_mds_tree(90, 100, 10, seed=4)
    assert not tree.children
    X, lam_bar, _ = V.fast_mds(Y, tree, 3, 10)
    Xc, lc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    assert np.max(np.abs(X - Xc)) < 1e-10 * np.max(np.abs(Xc))
    assert np.allclose(lam_bar, lc / 90, rtol=1e-12)


def err_fast_exact(fast=V.fast_mds, n=1500, l=200, s=20, seed=5):
    rng = np.random.default_rng(seed)
    Zc, Y = planted_rank_r(n, 4, 9, rng)
    tree = W.fast_mds_tree(n, l, s, seed, min_size=8)
    X, _, _ = fast(Y, tree, 4, s)
    return O.aligned_rel_error(X, Zc), tree


@pytest.mark.parametrize("n,depth", [(1500, 1), (5000, 2)])
def test_fast_exact_recovery(n, depth):
    e, tree = err_fast_exact(n=n)
    d = 0
    node = tree
    while node.children:
        d += 1
        node = max(node.children, key=lambda c: len(c.idx))
    assert d == depth
    assert e < 1e-10


def test_fast_leaf_variances():
    """Eq. (1) survives the alignments: each leaf's rows, after every
    Procrustes map above it, have covariance eigenvalues lambda^j / n_j."""
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((2000, 12)) * np.linspace(5, 1, 12)
    tree = W.fast_mds_tree(2000, 300, 25, seed=6, min_size=8)
    X, lam_bar, ex = V.fast_mds(Y, tree, 4, 25)
    for rows, lam in ex["leaves"]:
        Xl = X[rows]
        ev = np.sort(np.linalg.eigvalsh(np.cov(Xl.T, bias=True)))[::-1]
        assert np.max(np.abs(ev - lam / len(rows)) / (lam / len(rows))) < 1e-9
    assert np.allclose(lam_bar, np.mean([lam / len(rw) for rw, lam in ex["leaves"]], axis=0))


def test_planted_fast_transposed_map():
    def bad(Y, tree, r, s, rank_tol=1e-12):
        import oracle.variants as VV
        orig = VV.procrustes

        def proc(A, B):
            T, t = orig(A, B)
            return T.T, t
        VV.procrustes = proc
        try:
            return V.fast_mds(Y, tree, r, s, rank_tol)
        finally:
            VV.procrustes = orig
    e, _ = err_fast_exact(fast=bad)
    assert e > 1e-3
