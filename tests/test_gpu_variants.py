"""Parity of the GPU forms of the paper's other big-data MDS variants with
the CPU FP64 oracle (oracle/variants.py), through the C ABI.

MaxMin landmarks (Section 3.1, LMDS): the index list is an argmax sequence,
so it must equal the oracle's bit for bit -- on FP64, FP32 and byte rows,
with duplicated rows and exact ties (integer coordinates make the distances
exact on both sides).

Pivot MDS (Section 3.1): against the oracle's SVD of the n x l block of Q,
element by element (both apply the same sign convention) and after
alignment, FP64 at 1e-10 and FP32 at 1e-5, eigenvalue estimates at 1e-10 /
1e-6.

Fast MDS (Section 3.3): over the same random division tree as the oracle
(drawn on the host), one and two levels of division, against the oracle
after alignment at the same tolerances.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gb():
    from paper_2007_11919_gb300 import build
    build.build()
    import paper_2007_11919_gb300 as G
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return G


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ------------------------------------------------------------ MaxMin landmarks


@pytest.mark.parametrize("kind,n,d,l,first", [("f64", 3000, 20, 120, 17), ("f32", 5000, 100, 200, 0),
                                              ("f32", 2999, 7, 300, 2998), ("u8", 3000, 784, 150, 5),
                                              ("u8", 1000, 37, 64, 999), ("f64", 40, 3, 40, 0),
                                              ("f32", 4001, 48, 150, 7), ("u8", 2501, 64, 120, 3)])
def test_maxmin_bit_exact(gb, kind, n, d, l, first):
    if kind == "u8":
        Y = W.image_like(n, d, seed=n + d)
    else:
        Y = W.gaussian_dominant(n, d, min(5, d), seed=n + d, dtype=np.float64 if kind == "f64" else np.float32)
    want = O.maxmin_landmarks(Y, l, first)
    got = gb.mds_landmarks_maxmin(dev(Y), l, first).cpu().numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.uint8])
def test_maxmin_ties_and_duplicates(gb, dtype):
    """Integer lattice points, every one twice, in a shuffled order: many
    exact ties, broken by the lowest row index; once every point is covered
    the duplicates (distance 0) are chosen in index order; l = n takes every
    row exactly once."""
    g = np.stack(np.meshgrid(np.arange(7), np.arange(5), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
    Y3 = np.concatenate([g, g])[np.random.default_rng(1).permutation(2 * len(g))].astype(dtype)
    n = len(Y3)
    # d = 3 takes the general round; zero columns up to d = 16 (the same
    # distances) take the tiled round of FP32 and byte rows
    for Y in (Y3, np.concatenate([Y3, np.zeros((n, 13), dtype=dtype)], axis=1)):
        for l, first in ((n, 0), (60, 33), (n, n - 1)):
            want = O.maxmin_landmarks(Y, l, first)
            got = gb.mds_landmarks_maxmin(dev(Y), l, first).cpu().numpy()
            assert np.array_equal(got, want)
        assert sorted(gb.mds_landmarks_maxmin(dev(Y), n, 0).cpu().numpy()) == list(range(n))


def test_maxmin_full_size_prefix_and_gaps(gb):
    """n = 1,000,000 rows of the interpolation workload (d = 100 FP32),
    l = 1,000: the first picks equal the oracle's (a MaxMin sequence's prefix
    is the MaxMin sequence of that length), the picks are distinct, and the
    gap of each new pick to the earlier ones never grows."""
    w = W.INTERP_BF16
    Y = W.make_data(w, seed=0)
    idx = gb.mds_landmarks_maxmin(dev(Y), 1000, 123).cpu().numpy()
    assert len(set(idx.tolist())) == 1000
    assert np.array_equal(idx[:12], O.maxmin_landmarks(Y, 12, 123))
    D = O.sq_dist(Y[idx].astype(np.float64), Y[idx].astype(np.float64))
    gaps = np.array([D[k, :k].min() for k in range(1, 1000)])
    assert np.all(np.diff(gaps) <= 1e-9 * gaps[:-1])


def test_maxmin_then_interpolate(gb):
    """LMDS as the paper describes it: MaxMin landmarks, then Eq. (2) (Prop. 1:
    LMDS triangulation equals Gower's formula) -- against the oracle's
    interpolation MDS on the same landmarks."""
    Y = W.gaussian_dominant(4000, 30, 5, seed=8, dtype=np.float32)
    idx = gb.mds_landmarks_maxmin(dev(Y), 250, 0)
    X, var, _ = gb.mds_interpolate(dev(Y), idx, 5, "f32")
    Xo, vo, _ = O.interpolation_mds(Y, idx.cpu().numpy(), 5)
    assert O.aligned_rel_error(X.double().cpu().numpy(), Xo) < 1e-5
    assert np.max(np.abs(var.cpu().numpy() - vo) / vo) < 1e-6


def test_maxmin_argument_errors(gb):
    Y = dev(W.gaussian_dominant(100, 4, 2, seed=1))
    for l, first in ((0, 0), (101, 0), (10, 100), (10, -1)):
        with pytest.raises(gb.MdsError) as e:
            gb.mds_landmarks_maxmin(Y, l, first)
        assert e.value.status == 1


# ------------------------------------------------------------------- pivot MDS

PIV_TOL = {"f64": (1e-10, 1e-10), "f32": (1e-5, 1e-6)}


@pytest.mark.parametrize("prec,kind,n,d,l,r", [("f64", "f64", 1500, 10, 200, 3), ("f32", "f32", 2000, 100, 300, 10),
                                              ("f32", "u8", 1200, 784, 150, 5), ("f64", "f32", 999, 37, 129, 4),
                                              ("f32", "f64", 700, 130, 64, 16), ("f64", "u8", 500, 64, 500, 6)])
def test_pivot_matches_oracle(gb, prec, kind, n, d, l, r):
    """Ragged tiles (d = 10, 37, 130, 784), pivots = all points (l = n), FP64
    and FP32 arithmetic on FP64, FP32 and byte rows."""
    if kind == "u8":
        Y = W.image_like(n, d, seed=n + d)
    else:
        Y = W.gaussian_graded(n, d, seed=n + d, dtype=np.float64 if kind == "f64" else np.float32)
    piv = W.landmarks(n, l, seed=n + l)
    Xo, vo, lo = O.pivot_mds(Y, piv, r)
    X, var = gb.mds_pivot(dev(Y), dev(piv), r, prec)
    assert X.dtype == (torch.float64 if prec == "f64" else torch.float32)
    Xh = X.double().cpu().numpy()
    tx, tl = PIV_TOL[prec]
    assert np.max(np.abs(var.cpu().numpy() - vo) / vo) < tl
    assert O.aligned_rel_error(Xh, Xo) < tx
    assert np.max(np.abs(Xh - Xo)) < 10 * tx * np.max(np.abs(Xo))      # same sign convention


def test_pivot_two_copies_is_classical(gb):
    """A set made of two copies of a cloud with the pivots one copy: C C^T =
    (l/n) Q^2 exactly, so pivot MDS returns classical MDS of the set."""
    base = W.gaussian_graded(400, 12, seed=3, dtype=np.float64)
    Y = np.concatenate([base, base])
    X, var = gb.mds_pivot(dev(Y), dev(np.arange(400)), 4, "f64")
    Xc, lc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 4)
    assert O.aligned_rel_error(X.cpu().numpy(), Xc) < 1e-10
    assert np.allclose(var.cpu().numpy() * 800, lc, rtol=1e-10)


def test_pivot_argument_errors(gb):
    Y = dev(W.gaussian_graded(300, 5, seed=1, dtype=np.float32))
    with pytest.raises(gb.MdsError) as e:
        gb.mds_pivot(Y, dev(np.arange(50)), 6, "f32")                  # r > d
    assert e.value.status == 1
    with pytest.raises(gb.MdsError) as e:
        gb.mds_pivot(Y, dev(np.arange(50)), 3, "bf16")
    assert e.value.status == 7
    bad = np.arange(50)
    bad[7] = 300
    with pytest.raises(gb.MdsError) as e:
        gb.mds_pivot(Y, dev(bad), 3, "f32")
    assert e.value.status == 1


# -------------------------------------------------------------------- fast MDS

FAST_TOL = {"f64": (1e-10, 1e-10), "f32": (1e-5, 1e-6)}


@pytest.mark.parametrize("prec,n,d,l,s,r,depth", [("f64", 3000, 10, 500, 20, 3, 1), ("f32", 20_000, 50, 500, 40, 10, 2),
                                                  ("f32", 7001, 30, 500, 25, 5, 1), ("f64", 400, 8, 500, 20, 3, 0)])
def test_fast_matches_oracle(gb, prec, n, d, l, s, r, depth):
    """A tree of one or two levels of division (ragged last subsets), or a
    single leaf (n <= l: classical MDS)."""
    Y = W.gaussian_graded(n, d, seed=n + d, dtype=np.float64 if prec == "f64" else np.float32)
    tree = W.fast_mds_tree(n, l, s, seed=n)
    perm, rng, par = W.flatten_fast_tree(tree)
    got_depth = 0
    for k in range(len(par)):
        dk, x = 0, k
        while par[x] >= 0:
            x, dk = par[x], dk + 1
        got_depth = max(got_depth, dk)
    assert got_depth == depth
    Xo, lo, _ = O.fast_mds(Y, tree, r, s)
    X, var = gb.mds_fast(dev(Y), dev(perm), rng, par, s, r, prec)
    tx, tl = FAST_TOL[prec]
    assert np.max(np.abs(var.cpu().numpy() - lo) / lo) < tl
    assert O.aligned_rel_error(X.double().cpu().numpy(), Xo) < tx


def test_fast_exact_recovery(gb):
    """Points exactly in R^4 through two levels of division: the points up to
    one orthogonal map."""
    rng = np.random.default_rng(9)
    Z = rng.standard_normal((12_000, 4)) * np.array([6, 4, 3, 2.0])
    Y = Z @ np.linalg.qr(rng.standard_normal((9, 4)))[0].T
    tree = W.fast_mds_tree(12_000, 300, 15, seed=9)
    perm, rg, par = W.flatten_fast_tree(tree)
    X, _ = gb.mds_fast(dev(Y), dev(perm), rg, par, 15, 4, "f64")
    assert O.aligned_rel_error(X.cpu().numpy(), Z - Z.mean(axis=0)) < 1e-10


def test_fast_malformed_trees(gb):
    Y = dev(W.gaussian_graded(1000, 6, seed=1, dtype=np.float32))
    tree = W.fast_mds_tree(1000, 300, 20, seed=1)
    perm, rg, par = W.flatten_fast_tree(tree)
    bad_rng = rg.copy()
    bad_rng[1, 1] -= 1                                        # children no longer tile the root
    bad_par = par.copy()
    bad_par[2] = 2                                            # own parent
    for args in ((perm, bad_rng, par, 20, 3), (perm, rg, bad_par, 20, 3), (perm, rg, par, 3, 3),
                 (perm, rg, par, 400, 3)):
        with pytest.raises(gb.MdsError) as e:
            gb.mds_fast(Y, dev(args[0]), args[1], args[2], args[3], args[4], "f32")
        assert e.value.status == 1
