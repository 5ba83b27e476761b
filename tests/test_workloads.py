"""Host logic of the seeded input generators (shared by oracle and CUDA path)."""
import numpy as np

import workloads as W


def test_deterministic():
    a = W.gaussian_dominant(100, 7, 2, seed=3)
    b = W.gaussian_dominant(100, 7, 2, seed=3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, W.gaussian_dominant(100, 7, 2, seed=4))
    assert np.array_equal(W.landmarks(1000, 50, 1), W.landmarks(1000, 50, 1))


def test_dominant_variances():
    Y = W.gaussian_dominant(200_000, 6, 2, seed=0)
    v = Y.var(axis=0)
    assert np.allclose(v[:2], 15.0, rtol=0.02) and np.allclose(v[2:], 1.0, rtol=0.02)


def test_landmarks_distinct():
    idx = W.landmarks(1000, 300, 5)
    assert len(np.unique(idx)) == 300 and idx.min() >= 0 and idx.max() < 1000


def test_partitions_cover_once():
    for part in (W.partitions_uneven(100_000, 20, 800, 1200, 0), W.partitions_equal(10_000, 400, 50, 0)):
        allidx = np.concatenate([part.anchors, part.own])
        assert np.array_equal(np.sort(allidx), np.arange(len(allidx)))
        assert part.ptr[0] == 0 and part.ptr[-1] == len(part.own)
    part = W.partitions_uneven(100_000, 20, 800, 1200, 0)
    own = np.diff(part.ptr)
    assert own.min() >= 800 and own[:-1].max() <= 1200 and own[-1] < 2 * 1200
    assert np.array_equal(part.sizes(), own + 20)


def test_paper_part_count():
    """Section 3.2: p = ceil(1 + (n - l) / (l - c))."""
    n, l, c = 10_000, 400, 50
    part = W.partitions_equal(n, l, c, 0)
    assert part.p == int(np.ceil(1 + (n - l) / (l - c)))


def test_image_like_stats():
    Y = W.image_like(2000, 784, 0)
    assert Y.dtype == np.uint8
    z = (Y == 0).mean()
    assert 0.78 < z < 0.82
    nz = Y[Y > 0].astype(float)
    assert 150 < nz.mean() < 185 and nz.min() >= 1


def test_mixture_means():
    Y = W.gaussian_mixture(40_000, 10, 4, 5.0, 0, dtype=np.float64)
    m = Y.mean(axis=0)
    assert np.allclose(m[:4], 5.0 / np.sqrt(2) / 4, atol=0.05) and np.allclose(m[4:], 0, atol=0.05)


def test_serve_requests():
    t, s = W.serve_requests(1000, 1, 50_000, 100.0, 0)
    assert np.all(np.diff(t) > 0) and s.min() >= 1 and s.max() <= 50_000


def test_graded_variances_and_serve_sizes():
    Y = W.gaussian_graded(200_000, 14, seed=0)
    v = Y.var(axis=0)
    assert np.allclose(v[:10], 15.0 * 0.85 ** np.arange(10), rtol=0.03)
    assert np.allclose(v[10:], 1.0, rtol=0.03)
    t, sizes = W.serve_requests(20_000, *W.SERVE_SIZES, rate_per_s=1000.0, seed=0)
    assert np.all(np.diff(t) > 0) and sizes.min() >= 1 and sizes.max() <= 50_000
    # log-uniform sizes: mean (hi - lo) / ln(hi / lo) within sampling error
    assert abs(sizes.mean() / (50_000 / np.log(50_001)) - 1) < 0.05
    assert abs(len(t) / t[-1] / 1000.0 - 1) < 0.05


def test_fast_mds_tree():
    """Section 3.3's division: every row once, children partition their
    parent in order, leaves of at most l rows, p = floor(l / s) subsets of
    ceil(m / p) rows per split (one fewer after folding a small last one),
    and the same tree for the same seed."""
    n, l, s = 5000, 200, 20
    tree = W.fast_mds_tree(n, l, s, seed=3, min_size=8)
    assert np.array_equal(np.sort(tree.idx), np.arange(n))

    def walk(node):
        if not node.children:
            assert 0 < len(node.idx) <= l
            return
        m, p = len(node.idx), l // s
        assert len(node.idx) > l
        assert np.array_equal(node.idx, np.concatenate([c.idx for c in node.children]))
        assert len(node.children) in (p, p - 1)
        size = -(-m // p)
        assert all(len(c.idx) == size for c in node.children[:-1])
        assert max(s, 8) <= len(node.children[-1].idx) < size + max(s, 8)
        for c in node.children:
            walk(c)
    walk(tree)
    again = W.fast_mds_tree(n, l, s, seed=3, min_size=8)
    assert all(np.array_equal(a.idx, b.idx) for a, b in zip(tree.leaves(), again.leaves()))
    other = W.fast_mds_tree(n, l, s, seed=4, min_size=8)
    assert not np.array_equal(tree.leaves()[0].idx, other.leaves()[0].idx)
    assert not W.fast_mds_tree(150, l, s, seed=3).children
