"""Seeded synthetic inputs for interpolation MDS and divide-and-conquer MDS.

This module is the one thing the CPU oracle (``oracle/``) and the CUDA path
(``paper_2007_11919_gb300``) share: it draws data matrices, landmark subsets
and partitions, and holds none of the method's arithmetic (no distances, no
centering, no eigen-solves, no Procrustes).  Every random choice the method
makes (the random landmark subset of Section 3.1, the random connecting points
and random parts of Section 3.2) is drawn here and handed to both sides as
plain index arrays, so both compute on identical subsets.

Streams are numpy ``Philox`` generators keyed by ``(seed, stream id)``; the
same key gives the same numbers on x86-64 and aarch64 hosts.

Workload shapes follow the paper's simulation design (Section 4.1: rows drawn
from N(0, diag(15,...,15,1,...,1)), Euclidean distances) and stand in for the
EMNIST set of Section 5 with an image-like uint8 matrix of the same shape
(784 pixels in 0..255, mostly zeros), since the dataset itself is not used.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Stream ids: one independent Philox stream per purpose.
_S_DATA, _S_LANDMARK, _S_ANCHOR, _S_PART, _S_SIZE, _S_SERVE, _S_FAST = range(7)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, stream]))


# --------------------------------------------------------------------------- data


def gaussian_dominant(n: int, d: int, h: int, seed: int, var_dom: float = 15.0,
                      dtype=np.float64) -> np.ndarray:
    """n x d rows from N(0, diag(var_dom x h, 1 x (d-h))) (Section 4.1)."""
    g = _rng(seed, _S_DATA)
    sd = np.ones(d)
    sd[:h] = math.sqrt(var_dom)
    out = np.empty((n, d), dtype=dtype)
    step = max(1, (1 << 22) // max(d, 1))
    for i in range(0, n, step):
        j = min(n, i + step)
        out[i:j] = g.standard_normal((j - i, d)) * sd
    return out


def gaussian_mixture(n: int, d: int, k: int, spacing: float, seed: int,
                     dtype=np.float32) -> np.ndarray:
    """Equal-weight mixture of k unit-covariance Gaussians in R^d.

    The k means form a regular simplex with pairwise distance ``spacing``:
    mu_c = (spacing / sqrt(2)) e_c, c = 0..k-1.
    """
    g = _rng(seed, _S_DATA)
    out = np.empty((n, d), dtype=dtype)
    a = spacing / math.sqrt(2.0)
    step = max(1, (1 << 22) // max(d, 1))
    for i in range(0, n, step):
        j = min(n, i + step)
        blk = g.standard_normal((j - i, d))
        comp = g.integers(0, k, size=j - i)
        blk[np.arange(j - i), comp] += a
        out[i:j] = blk
    return out


def gaussian_graded(n: int, d: int, seed: int, top: int = 10, var_top: float = 15.0,
                    decay: float = 0.85, dtype=np.float32) -> np.ndarray:
    """n x d rows from N(0, diag(s)) with s_k = var_top * decay^k for the first
    ``top`` coordinates and 1 for the rest: distinct leading variances, so the
    top-r principal subspace is well separated for every r <= top."""
    g = _rng(seed, _S_DATA)
    sd = np.ones(d)
    k = min(top, d)
    sd[:k] = np.sqrt(var_top * decay ** np.arange(k))
    out = np.empty((n, d), dtype=dtype)
    step = max(1, (1 << 22) // max(d, 1))
    for i in range(0, n, step):
        j = min(n, i + step)
        out[i:j] = g.standard_normal((j - i, d)) * sd
    return out


def image_like(n: int, d: int, seed: int, zero_frac: float = 0.8,
               mean: float = 180.0, sd: float = 60.0) -> np.ndarray:
    """n x d uint8 'pixels': a fraction ``zero_frac`` are 0, the rest are
    round(clip(N(mean, sd), 1, 255)); pixels are i.i.d."""
    g = _rng(seed, _S_DATA)
    out = np.empty((n, d), dtype=np.uint8)
    step = max(1, (1 << 21) // max(d, 1))
    for i in range(0, n, step):
        j = min(n, i + step)
        v = np.rint(np.clip(g.normal(mean, sd, size=(j - i, d)), 1.0, 255.0))
        v[g.random((j - i, d)) < zero_frac] = 0.0
        out[i:j] = v.astype(np.uint8)
    return out


# ---------------------------------------------------------------- random subsets


def landmarks(n: int, l: int, seed: int) -> np.ndarray:
    """A uniformly random l-subset of range(n), as int64, in draw order."""
    if not 0 < l <= n:
        raise ValueError("need 0 < l <= n")
    return _rng(seed, _S_LANDMARK).permutation(n)[:l].astype(np.int64)


@dataclasses.dataclass
class Partitioning:
    """Divide-and-conquer layout.

    ``anchors`` (c,) are the connecting points shared by every part;
    part j owns ``own[ptr[j]:ptr[j+1]]``; the points of part j are
    ``anchors`` followed by its own points, so n_j = c + own_j.
    Every index in range(n) is either an anchor or owned by exactly one part.
    """
    anchors: np.ndarray
    ptr: np.ndarray
    own: np.ndarray

    @property
    def p(self) -> int:
        return len(self.ptr) - 1

    @property
    def c(self) -> int:
        return len(self.anchors)

    def sizes(self) -> np.ndarray:
        """n_j, the number of points of each part (anchors included)."""
        return np.diff(self.ptr) + self.c

    def members(self, j: int) -> np.ndarray:
        return np.concatenate([self.anchors, self.own[self.ptr[j]:self.ptr[j + 1]]])


def partitions_uneven(n: int, c: int, own_lo: int, own_hi: int, seed: int) -> Partitioning:
    """c random connecting points; the other n-c points in random order are cut
    into parts whose own sizes are drawn uniformly from [own_lo, own_hi].  A
    last remainder smaller than own_lo is folded into the part before it."""
    if c >= n:
        raise ValueError("need c < n")
    perm = _rng(seed, _S_ANCHOR).permutation(n).astype(np.int64)
    anchors, rest = perm[:c], perm[c:]
    rest = rest[_rng(seed, _S_PART).permutation(len(rest))]
    gs = _rng(seed, _S_SIZE)
    sizes = []
    left = len(rest)
    while left > 0:
        s = int(gs.integers(own_lo, own_hi + 1))
        s = min(s, left)
        sizes.append(s)
        left -= s
    if len(sizes) > 1 and sizes[-1] < own_lo:
        tail = sizes.pop()
        sizes[-1] += tail
    ptr = np.zeros(len(sizes) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(sizes)
    return Partitioning(anchors=anchors, ptr=ptr, own=rest)


def partitions_equal(n: int, l: int, c: int, seed: int) -> Partitioning:
    """The paper's own layout (Section 3.2): parts of l points (c shared
    connecting points + l-c own points), p = ceil(1 + (n-l)/(l-c)); the last
    part may be smaller."""
    if not c < l:
        raise ValueError("need c < l")
    perm = _rng(seed, _S_ANCHOR).permutation(n).astype(np.int64)
    anchors, rest = perm[:c], perm[c:]
    rest = rest[_rng(seed, _S_PART).permutation(len(rest))]
    own = l - c
    nparts = max(1, math.ceil(len(rest) / own))
    ptr = np.minimum(np.arange(nparts + 1, dtype=np.int64) * own, len(rest))
    return Partitioning(anchors=anchors, ptr=ptr, own=rest)


@dataclasses.dataclass
class FastNode:
    """One node of fast MDS's random division (Section 3.3).

    ``idx`` are the node's points; an inner node's ``children`` partition
    ``idx`` in order (idx = concatenation of the children's idx), and the
    first ``s`` points of each child are its sampling points."""
    idx: np.ndarray
    children: list

    def leaves(self):
        if not self.children:
            return [self]
        return [leaf for ch in self.children for leaf in ch.leaves()]


def fast_mds_tree(n: int, l: int, s: int, seed: int, min_size: int = 0) -> FastNode:
    """Fast MDS's recursive random division (Section 3.3) of range(n): a node
    of m > l points is split, in a random order, into p = floor(l / s)
    subsets of ceil(m / p) points (the last one smaller; a last subset of
    fewer than max(s, min_size) points is folded into the one before it),
    and each subset larger than l is divided again.  Each split draws its
    own permutation from a Philox stream keyed by (seed, split number in
    depth-first order)."""
    p = l // s
    if p < 2:
        raise ValueError("need l >= 2 s so that a division makes progress")
    counter = [0]

    def build(idx):
        m = len(idx)
        if m <= l:
            return FastNode(idx, [])
        g = np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF,
                                                     (_S_FAST << 32) | counter[0]]))
        counter[0] += 1
        perm = idx[g.permutation(m)]
        size = -(-m // p)
        cuts = [perm[i:i + size] for i in range(0, m, size)]
        if len(cuts) > 1 and len(cuts[-1]) < max(s, min_size):
            tail = cuts.pop()
            cuts[-1] = np.concatenate([cuts[-1], tail])
        children = [build(c) for c in cuts]
        return FastNode(np.concatenate([ch.idx for ch in children]), children)

    return build(np.arange(n, dtype=np.int64))


def flatten_fast_tree(tree: FastNode):
    """The division tree as flat arrays for the C ABI: perm (the root's
    points in order; every node's points are a contiguous range of it),
    node_range (nnodes x 2: [begin, end) in perm) and node_parent (-1 for the
    root, node 0), nodes numbered depth first."""
    ranges, parents = [], []

    def visit(node, begin, parent):
        k = len(ranges)
        ranges.append((begin, begin + len(node.idx)))
        parents.append(parent)
        at = begin
        for ch in node.children:
            visit(ch, at, k)
            at += len(ch.idx)

    visit(tree, 0, -1)
    return (np.asarray(tree.idx, dtype=np.int64), np.asarray(ranges, dtype=np.int64),
            np.asarray(parents, dtype=np.int32))


# -------------------------------------------------------------------- serving


def serve_requests(count: int, lo: int, hi: int, rate_per_s: float, seed: int):
    """Poisson arrivals: (arrival time [s], size) pairs; sizes are
    floor(exp(U(ln lo, ln(hi+1)))) clipped to [lo, hi] (log-uniform)."""
    g = _rng(seed, _S_SERVE)
    t = np.cumsum(g.exponential(1.0 / rate_per_s, size=count))
    sizes = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi + 1), size=count)))
    sizes = np.clip(sizes, lo, hi).astype(np.int64)
    return t, sizes


# ------------------------------------------------------------- named workloads


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "interp", "dc", "affine", "maxmin", "pivot", "fast", "serve"
    n: int
    d: int
    r: int
    prec: str          # distance precision: "f64", "f32", "bf16", "fp8"
    l: int = 0         # landmarks (interp) / part size (equal dc)
    c: int = 0         # connecting points (dc); sampling points s (fast)
    own_lo: int = 0
    own_hi: int = 0


# The five workloads of this project; names say what they are.
CLASSICAL_INTERP_F64 = Workload("interp_f64_n2000_d10_l300_r3", "interp", 2000, 10, 3, "f64", l=300)
DC_F32 = Workload("dc_f32_n100000_d100_parts800-1200_c20_r10", "dc", 100_000, 100, 10, "f32",
                  c=20, own_lo=800, own_hi=1200)
INTERP_BF16 = Workload("interp_bf16_n1000000_d100_l1000_r10", "interp", 1_000_000, 100, 10, "bf16",
                       l=1000)
# The same interpolation problem on the plain FP32 path (SIMT distance tiles
# and projection, one problem): the baseline the mixed-precision forms are
# compared against.
INTERP_F32 = Workload("interp_f32_n1000000_d100_l1000_r10", "interp", 1_000_000, 100, 10, "f32",
                      l=1000)
# The same data by the affine form of Eq. (2) (rows given by coordinates): one
# pass over Y after the landmark eigenproblem.
INTERP_AFFINE_F32 = Workload("affine_f32_n1000000_d100_l1000_r10", "affine", 1_000_000, 100, 10, "f32",
                             l=1000)
SERVE_BF16 = Workload("serve_bf16_d100_l500r2_l1000r5_l2000r10_req1-50000", "serve", 200_000, 100, 10,
                      "bf16", l=2000)
# Resident models of the serving workload: (landmarks, r).
SERVE_MODELS = ((500, 2), (1000, 5), (2000, 10))
SERVE_SIZES = (1, 50_000)
# The paper's other variants at the interpolation workload's scale: MaxMin
# landmarks (LMDS) on the mixture data; pivot MDS and fast MDS on rows with
# distinct leading variances (N(0, diag(15 * 0.85^k, k < 10; 1 ...))), so that
# every subset's top-10 subspace is well separated.
MAXMIN_F32 = Workload("maxmin_f32_n1000000_d100_l1000", "maxmin", 1_000_000, 100, 10, "f32", l=1000)
PIVOT_F32 = Workload("pivot_f32_n1000000_d100_graded_l1000_r10", "pivot", 1_000_000, 100, 10, "f32", l=1000)
FAST_F32 = Workload("fast_f32_n1000000_d100_graded_l1000_s20_r10", "fast", 1_000_000, 100, 10, "f32", l=1000,
                    c=20)
IMAGE_FP8 = Workload("image_fp8_n814255_d784_l2000_r10", "interp", 814_255, 784, 10, "fp8", l=2000,
                     c=50)
# The same image-like set by divide-and-conquer: parts of l = 2000 points with
# c = 50 shared connecting points (Section 3.2 layout), FP8 nibble distance tiles.
IMAGE_DC = Workload("image_dc_fp8_n814255_d784_parts2000_c50_r10", "dc", 814_255, 784, 10, "fp8", l=2000,
                    c=50)


def make_data(w: Workload, seed: int, n: int | None = None) -> np.ndarray:
    """Data matrix of workload ``w`` (optionally only its first n rows)."""
    n = w.n if n is None else n
    if w is CLASSICAL_INTERP_F64 or w.name == CLASSICAL_INTERP_F64.name:
        return gaussian_dominant(n, w.d, 3, seed, dtype=np.float64)
    if w.name == DC_F32.name:
        return gaussian_dominant(n, w.d, 5, seed, dtype=np.float32)
    if w.name in (INTERP_BF16.name, INTERP_F32.name, INTERP_AFFINE_F32.name, MAXMIN_F32.name):
        return gaussian_mixture(n, w.d, 4, 5.0, seed, dtype=np.float32)
    if w.name in (SERVE_BF16.name, PIVOT_F32.name, FAST_F32.name):
        return gaussian_graded(n, w.d, seed)
    if w.name in (IMAGE_FP8.name, IMAGE_DC.name):
        return image_like(n, w.d, seed)
    raise KeyError(w.name)
