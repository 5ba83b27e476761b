"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (relative Frobenius error after the best orthogonal alignment,
Section 4.1's Procrustes comparison):
  FP64 path                 1e-10   (eigenvalues 1e-10 relative)
  FP32 path                 1e-5    (eigenvalues 1e-6 relative)
  BF16 / FP8 distance path  2e-3    (eigenvalues 1e-6 relative)
"""
import multiprocessing
import os

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-5, "bf16": 2e-3}
LAM_TOL = {"f64": 1e-10, "f32": 1e-6, "bf16": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def gb():
    from paper_2007_11919_gb300 import build
    build.build()
    import paper_2007_11919_gb300 as G
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return G


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))


# ------------------------------------------------------------- classical


@pytest.mark.parametrize("n,d,r", [(300, 10, 3), (64, 5, 2), (129, 40, 6)])
def test_classical_f64(gb, n, d, r):
    Y = W.gaussian_dominant(n, d, r, seed=n)
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), r)
    X, lam = gb.mds_classical(dev(Y), r, "f64")
    assert rel(host(lam), lo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]
    # same sign convention on both sides: elementwise agreement
    assert np.max(np.abs(host(X) - Xo)) < 1e-8 * np.max(np.abs(Xo))


def test_classical_dist_non_euclidean(gb):
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((257, 6)) * np.array([5, 4, 3, 2, 1, 1.0])
    D = O.sq_dist(Y, Y)
    E = rng.uniform(0, 0.5, size=D.shape)
    D = D + E + E.T
    np.fill_diagonal(D, 0.0)
    Xo, lo, _, _ = O.classical_mds(D, 4)
    X, lam = gb.mds_classical_dist(dev(D), 4)
    assert rel(host(lam), lo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]


def test_classical_f32(gb):
    Y = W.gaussian_dominant(500, 20, 4, seed=5, dtype=np.float32)
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), 4)
    X, lam = gb.mds_classical(dev(Y), 4, "f32")
    assert X.dtype == torch.float32
    assert rel(host(lam), lo) < LAM_TOL["f32"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f32"]


def test_classical_uint8(gb):
    Y = W.image_like(300, 64, seed=2)
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), 5)
    X, lam = gb.mds_classical(dev(Y), 5, "f64")
    assert rel(host(lam), lo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]


@pytest.mark.parametrize("cluster", [1, 2, 3, 8, 16])
def test_cluster_sizes_agree(gb, cluster):
    Y = W.gaussian_dominant(1000, 30, 5, seed=9)
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), 5)
    X, lam = gb.mds_classical(dev(Y), 5, "f64", cluster=cluster)
    assert rel(host(lam), lo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]


@pytest.mark.parametrize("n,cluster", [(500, 3), (500, 4), (500, 5), (500, 8), (500, 16), (1021, 3),
                                       (1021, 6), (1021, 7), (130, 5), (130, 16), (2050, 8), (1100, 3),
                                       (1500, 4), (2050, 5), (2050, 16), (3001, 9), (4000, 16)])
def test_symmetric_ranges_classical_f32(gb, n, cluster):
    """FP32 Q in one cluster: the symmetric ranges (each off-diagonal block of
    Q read once, used for both triangles) against the oracle and against the
    whole-row matvec, for odd and even cluster sizes, ranges that wrap, and
    sizes where the ranges are not used (too few rows per CTA; ranges longer
    than one stage: n = 1,100 ... 4,000)."""
    Y = W.gaussian_dominant(n, 30, 5, seed=n + cluster, dtype=np.float32)
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), 5)
    X, lam = gb.mds_classical(dev(Y), 5, "f32", cluster=cluster)
    Xf, lamf = gb.mds_classical(dev(Y), 5, "f32", cluster=cluster, full_matvec=True)
    for Xg, lg in ((X, lam), (Xf, lamf)):
        assert rel(host(lg), lo) < LAM_TOL["f32"]
        assert O.aligned_rel_error(host(Xg), Xo) < TOL["f32"]
    assert rel(host(lam), host(lamf)) < 1e-6


def test_tiny_problems(gb):
    Y = W.gaussian_dominant(5, 4, 3, seed=1)                   # n = r + 2
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    X, lam = gb.mds_classical(dev(Y), 3, "f64")
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]
    Y1 = np.random.default_rng(0).standard_normal((40, 1))     # d = 1, r = 1
    Xo1, lo1, _, _ = O.classical_mds(O.sq_dist(Y1, Y1), 1)
    X1, l1 = gb.mds_classical(dev(Y1), 1, "f64")
    assert O.aligned_rel_error(host(X1), Xo1) < TOL["f64"] and rel(host(l1), lo1) < 1e-10


def test_rank_error(gb):
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((80, 2)) @ rng.standard_normal((2, 6))   # rank 2
    with pytest.raises(gb.MdsError) as e:
        gb.mds_classical(dev(Y), 3, "f64")
    assert e.value.status == 4


# ---------------------------------------------------------- interpolation


def test_interp_f64_small_config(gb):
    """n=2,000 points in d=10, N(0, diag(15,15,15,1,...)), l=300, r=3, FP64."""
    w = W.CLASSICAL_INTERP_F64
    Y = W.make_data(w, seed=0)
    idx = W.landmarks(w.n, w.l, seed=0)
    Xo, vo, _ = O.interpolation_mds(Y, idx, w.r)
    X, var, _ = gb.mds_interpolate(dev(Y), dev(idx), w.r, "f64")
    assert rel(host(var), vo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]
    assert np.max(np.abs(host(X) - Xo)) < 1e-8 * np.max(np.abs(Xo))


@pytest.mark.parametrize("n,l", [(5000, 500), (3001, 130)])
def test_interp_f32(gb, n, l):
    Y = W.gaussian_dominant(n, 100, 10, seed=l, dtype=np.float32)
    idx = W.landmarks(n, l, seed=l)
    Xo, vo, _ = O.interpolation_mds(Y, idx, 10)
    X, var, _ = gb.mds_interpolate(dev(Y), dev(idx), 10, "f32")
    assert rel(host(var), vo) < LAM_TOL["f32"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f32"]


def test_interp_bf16(gb):
    Y = W.gaussian_mixture(8000, 100, 4, 5.0, seed=1)
    idx = W.landmarks(8000, 1000, seed=1)
    Xo, vo, _ = O.interpolation_mds(Y, idx, 10)
    X, var, _ = gb.mds_interpolate(dev(Y), dev(idx), 10, "bf16")
    assert rel(host(var), vo) < LAM_TOL["bf16"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["bf16"]


def test_interp_l_equals_n_is_classical(gb):
    Y = W.gaussian_dominant(200, 8, 3, seed=4)
    idx = np.arange(200)
    X, var, _ = gb.mds_interpolate(dev(Y), dev(idx), 3, "f64")
    Xc, lc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    assert O.aligned_rel_error(host(X), Xc) < TOL["f64"]
    assert rel(host(var) * 200, lc) < 1e-10


def test_interp_full_size_sampled(gb):
    """n=1,000,000, d=100 mixture, l=1,000, r=10, BF16 distances: sampled rows
    against the oracle (landmark MDS + Eq. (2) for each sampled row)."""
    w = W.INTERP_BF16
    Y = W.make_data(w, seed=0)
    idx = W.landmarks(w.n, w.l, seed=0)
    X, var, _ = gb.mds_interpolate(dev(Y), dev(idx), w.r, "bf16")
    Xh = host(X)
    L = Y[idx].astype(np.float64)
    D1 = O.sq_dist(L, L)
    X1, lam, _, _ = O.classical_mds(D1, w.r)
    rng = np.random.default_rng(0)
    rows = np.setdiff1d(rng.choice(w.n, 3000, replace=False), idx)
    Xs = O.gower_interpolate(X1, lam, D1, O.sq_dist(Y[rows], L))
    both = np.vstack([Xh[rows], Xh[idx]])
    ref = np.vstack([Xs, X1])
    assert O.aligned_rel_error(both, ref) < TOL["bf16"]
    assert rel(host(var), lam / w.l) < LAM_TOL["bf16"]
    assert np.all(np.isfinite(Xh))


@pytest.mark.parametrize("prec,kind,n,d,l,r", [("f64", "f64", 3000, 20, 300, 5), ("f32", "f32", 5000, 100, 1000, 10),
                                              ("f32", "u8", 2000, 64, 250, 6), ("f64", "f32", 777, 9, 129, 3),
                                              ("f32", "f64", 2500, 30, 200, 4), ("f64", "u8", 1500, 64, 180, 5)])
def test_interp_affine(gb, prec, kind, n, d, l, r):
    """Affine form of Eq. (2) for coordinate rows: the oracle's affine form
    and its distance form (Gower) agree with the GPU result."""
    if kind == "u8":
        Y = W.image_like(n, d, seed=n)
    else:
        Y = W.gaussian_dominant(n, d, r, seed=n, dtype=np.float64 if kind == "f64" else np.float32)
    idx = W.landmarks(n, l, seed=n)
    Xo, vo, _ = O.affine_interpolation(Y, idx, r)
    Xg, _, _ = O.interpolation_mds(Y, idx, r)
    X, var = gb.mds_interpolate_affine(dev(Y), dev(idx), r, prec)
    assert X.dtype == (torch.float64 if prec == "f64" else torch.float32)
    assert rel(host(var), vo) < LAM_TOL[prec]
    assert O.aligned_rel_error(host(X), Xo) < TOL[prec]
    assert O.aligned_rel_error(host(X), Xg) < TOL[prec]


@pytest.mark.parametrize("n,d,l,r", [(1001, 8, 120, 3), (4097, 100, 400, 1), (3000, 64, 300, 15),
                                     (2000, 128, 250, 16), (999, 4, 100, 2), (5003, 36, 333, 7)])
def test_interp_affine_f32_tile_shapes(gb, n, d, l, r):
    """The FP32 pass over Y at row widths whose tiles come as one copy (d/4
    odd) or one copy per row (d/4 even), odd and even r, ragged last tiles;
    the same rows at a base that is not 16-byte aligned take the general
    kernel and give the same embedding."""
    Y = W.gaussian_dominant(n, d, min(r, d), seed=d + r, dtype=np.float32)
    idx = W.landmarks(n, l, seed=n)
    Xo, vo, _ = O.affine_interpolation(Y, idx, r)
    X, var = gb.mds_interpolate_affine(dev(Y), dev(idx), r, "f32")
    assert rel(host(var), vo) < LAM_TOL["f32"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f32"]
    buf = torch.zeros(n * d + 1, dtype=torch.float32, device="cuda")
    buf[1:] = dev(Y).reshape(-1)
    Xu, _ = gb.mds_interpolate_affine(buf[1:].view(n, d), dev(idx), r, "f32")
    assert np.linalg.norm(host(Xu) - host(X)) < 1e-6 * np.linalg.norm(host(X))


def test_interp_affine_all_landmarks_and_errors(gb):
    """l = n: every row is a landmark, the result is classical MDS; BF16
    is not offered for the affine form."""
    Y = W.gaussian_dominant(400, 8, 3, seed=2)
    Xc, lc, _, _ = O.classical_mds(O.sq_dist(Y, Y), 3)
    X, var = gb.mds_interpolate_affine(dev(Y), dev(np.arange(400)), 3, "f64")
    assert O.aligned_rel_error(host(X), Xc) < TOL["f64"]
    assert rel(host(var), lc / 400) < LAM_TOL["f64"]
    with pytest.raises(gb.MdsError):
        gb.mds_interpolate_affine(dev(Y.astype(np.float32)), dev(np.arange(50)), 3, "bf16")


def test_bad_landmark_index(gb):
    Y = W.gaussian_dominant(500, 10, 3, seed=2)
    idx = W.landmarks(500, 100, seed=2)
    idx[17] = 500                                           # out of range
    with pytest.raises(gb.MdsError) as e:
        gb.mds_interpolate(dev(Y), dev(idx), 3, "f64")
    assert e.value.status == 1


def test_workspace_too_small(gb):
    Y = dev(W.gaussian_dominant(500, 10, 3, seed=2))
    idx = dev(W.landmarks(500, 100, seed=2))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    # pass an explicit, too-small workspace through the raw ABI
    import ctypes
    from paper_2007_11919_gb300.mds import MdsOpts, _lib
    o = MdsOpts(prec=0, stream=ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                workspace=ctypes.c_void_p(ws.data_ptr()), workspace_bytes=1024)
    X = torch.empty((500, 3), dtype=torch.float64, device="cuda")
    v = torch.empty(3, dtype=torch.float64, device="cuda")
    s = _lib().mds_interpolate(ctypes.c_void_p(Y.data_ptr()), 0, 500, 10, ctypes.c_void_p(idx.data_ptr()),
                               100, 3, ctypes.byref(o), ctypes.c_void_p(X.data_ptr()),
                               ctypes.c_void_p(v.data_ptr()), None)
    assert s == 8


# ------------------------------------------------------ embed / model


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_embed_new_matches_interpolate(gb, prec, tmp_path):
    dt = np.float64 if prec == "f64" else np.float32
    Y = W.gaussian_dominant(3000, 50, 5, seed=11, dtype=dt)
    idx = W.landmarks(3000, 400, seed=11)
    X, var, model = gb.mds_interpolate(dev(Y), dev(idx), 5, prec, want_model=True)
    info = model.info()
    assert info["l"] == 400 and info["r"] == 5 and info["prec"] == prec
    Xe = gb.mds_embed_new(model, dev(Y))
    rest = np.setdiff1d(np.arange(3000), idx)
    # the same kernel computes both: bitwise equal on non-landmark rows
    assert torch.equal(Xe[rest], X[rest])
    # landmarks interpolate onto themselves (Gower's formula reproduces X_1)
    assert O.aligned_rel_error(host(Xe[idx]), host(X[idx])) < 10 * TOL[prec]
    # each row alone equals the row in a batch
    one = gb.mds_embed_new(model, dev(Y[rest[5:6]]))
    assert torch.equal(one[0], X[rest[5]])
    path = str(tmp_path / "m.gbmds")
    model.save(path)
    m2 = gb.Model.load(path)
    assert torch.equal(gb.mds_embed_new(m2, dev(Y[:100])), Xe[:100])


# ------------------------------------------------------ divide-and-conquer


def test_dc_f64_small(gb):
    Y = W.gaussian_dominant(3000, 10, 3, seed=3)
    part = W.partitions_uneven(3000, 10, 300, 420, seed=3)
    Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 3)
    X, var = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), 3, "f64")
    assert rel(host(var), lo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]


@pytest.mark.parametrize("r", [1, 2, 7, 11, 16, 17, 32])
def test_dc_f64_target_dimensions(gb, r):
    """Procrustes packs floor(32 / r) column pairs into a warp: r = 1 (a
    dummy column only), odd r, r just past a packing boundary (11, 17) and the
    largest r (one pair per warp), FP64 against the oracle."""
    Y = W.gaussian_dominant(2400, 40, min(r, 40), seed=r, var_dom=30.0)
    part = W.partitions_uneven(2400, 40, 300, 420, seed=r)
    Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, r)
    X, var = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), r, "f64")
    assert rel(host(var), lo) < LAM_TOL["f64"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]


def test_dc_f32(gb):
    Y = W.gaussian_dominant(12_000, 100, 5, seed=4, dtype=np.float32)
    part = W.partitions_uneven(12_000, 20, 800, 1200, seed=4)
    Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 10)
    X, var = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), 10, "f32")
    assert rel(host(var), lo) < LAM_TOL["f32"]
    assert O.aligned_rel_error(host(X), Xo) < TOL["f32"]


@pytest.mark.parametrize("cluster", [3, 4, 5, 8])
def test_dc_f32_symmetric_ranges(gb, cluster):
    """D&C parts of uneven sizes at a fixed cluster size: symmetric ranges and
    whole rows both match the oracle."""
    Y = W.gaussian_dominant(6_000, 100, 5, seed=cluster, dtype=np.float32)
    part = W.partitions_uneven(6_000, 20, 800, 1200, seed=cluster)
    Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 10)
    for full in (False, True):
        X, var = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), 10, "f32",
                                       cluster=cluster, full_matvec=full)
        assert rel(host(var), lo) < LAM_TOL["f32"]
        assert O.aligned_rel_error(host(X), Xo) < TOL["f32"]
        st = gb.mds.mds_last_stats()
        # streamed bytes: whole rows, or about (cs + 1) / (2 cs) of them for
        # the parts whose ranges fit a stage (the last, largest part may not)
        ratio = st["eig_qread"] / st["eig_qbytes"]
        if full:
            assert ratio == pytest.approx(1.0, rel=1e-2)
        else:
            assert (cluster + 1) / (2 * cluster) - 0.01 < ratio < 0.95


def test_dc_exact_rank_r(gb):
    """Points exactly in R^4: D&C returns them up to one orthogonal map."""
    rng = np.random.default_rng(8)
    Z = rng.standard_normal((4000, 4)) * np.array([6, 4, 3, 2.0])
    Y = Z @ np.linalg.qr(rng.standard_normal((9, 4)))[0].T
    part = W.partitions_uneven(4000, 12, 500, 700, seed=8)
    X, _ = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), 4, "f64")
    assert O.aligned_rel_error(host(X), Z - Z.mean(axis=0)) < 1e-10


def test_dc_full_size_sampled(gb):
    """n=100,000, d=100, parts of 800-1,200 own points + 20 connecting points,
    r=10, FP32: parts 0, 1, p/2 and p-1 against the oracle."""
    w = W.DC_F32
    Y = W.make_data(w, seed=0)
    part = W.partitions_uneven(w.n, w.c, w.own_lo, w.own_hi, seed=0)
    X, var = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), w.r, "f32")
    Xh = host(X)
    rows, ref = [], []
    for j in sorted({0, 1, part.p // 2, part.p - 1}):
        rj, Xj, _ = O.divide_conquer_part(Y, part.anchors, part.ptr, part.own, j, w.r)
        rows.append(rj)
        ref.append(Xj)
    rows = np.concatenate(rows)
    assert O.aligned_rel_error(Xh[rows], np.vstack(ref)) < TOL["f32"]
    assert np.all(np.isfinite(Xh)) and np.all(host(var) > 0)


def test_dc_deterministic(gb):
    Y = dev(W.gaussian_dominant(5000, 20, 4, seed=6, dtype=np.float32))
    part = W.partitions_uneven(5000, 10, 600, 900, seed=6)
    a = gb.mds_divide_conquer(Y, dev(part.anchors), part.ptr, dev(part.own), 4, "f32")[0]
    b = gb.mds_divide_conquer(Y, dev(part.anchors), part.ptr, dev(part.own), 4, "f32")[0]
    assert torch.equal(a, b)


# ------------------------------------------- tensor-core Gower (BF16 split)


@pytest.mark.parametrize("n,d,l,r", [(200, 16, 130, 3), (1000, 100, 256, 10), (777, 64, 129, 16),
                                     (4000, 128, 1000, 10), (130, 8, 128, 1)])
def test_bf16_tensor_core_embed(gb, n, d, l, r):
    """embed_new on the tcgen05 path (ragged tiles and chunks, one and two K
    atoms, r = 1..16) against Eq. (2) on the same landmark model."""
    Y = W.gaussian_mixture(n + l, d, 4, 5.0, seed=d + l, dtype=np.float32)
    idx = np.arange(n, n + l)
    X, var, model = gb.mds_interpolate(dev(Y), dev(idx), r, "bf16", want_model=True)
    L = Y[idx].astype(np.float64)
    D1 = O.sq_dist(L, L)
    X1, lam, _, _ = O.classical_mds(D1, r)
    Xo = O.gower_interpolate(X1, lam, D1, O.sq_dist(Y[:n], L))
    Xe = host(gb.mds_embed_new(model, dev(Y[:n])))
    assert np.all(np.isfinite(Xe))
    assert O.aligned_rel_error(Xe, Xo) < TOL["bf16"]
    assert O.aligned_rel_error(host(X)[:n], Xo) < TOL["bf16"]


# ------------------------------------------------- byte rows on the tensor cores


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("n,d,l,r", [(3000, 784, 300, 10), (1000, 100, 257, 5), (777, 37, 129, 3),
                                     (300, 784, 256, 16)])
def test_u8_tensor_core_interp(gb, prec, n, d, l, r, tmp_path):
    """Image-like byte rows: exact BF16 operands or exact E4M3 nibble planes on
    tcgen05 (ragged tiles, ragged landmark chunks, d not a multiple of 16)."""
    Y = W.image_like(n, d, seed=d + l)
    idx = W.landmarks(n, l, seed=n + r)
    X, var, model = gb.mds_interpolate(dev(Y), dev(idx), r, prec, want_model=True)
    Xo, vo, _ = O.interpolation_mds(Y.astype(np.float64), idx, r)
    err = O.aligned_rel_error(host(X), Xo)
    assert err < TOL["bf16"], err
    assert rel(host(var), vo) < LAM_TOL["f32"]
    rest = np.setdiff1d(np.arange(n), idx)
    Xe = gb.mds_embed_new(model, dev(Y))
    assert torch.equal(Xe[rest], X[rest])
    path = str(tmp_path / "u8.gbmds")
    model.save(path)
    m2 = gb.Model.load(path)
    assert torch.equal(gb.mds_embed_new(m2, dev(Y[:50])), Xe[:50])
    with pytest.raises(gb.MdsError):
        gb.mds_embed_new(model, dev(Y[:50].astype(np.float32)))


def test_u8_bf16_and_fp8_agree(gb):
    """Both encodings give exact products: the two projections agree far
    below the BF16 / FP8 tolerance."""
    Y = W.image_like(5000, 784, seed=5)
    idx = W.landmarks(5000, 500, seed=5)
    Xb, _, _ = gb.mds_interpolate(dev(Y), dev(idx), 10, "bf16")
    Xf, _, _ = gb.mds_interpolate(dev(Y), dev(idx), 10, "fp8")
    scale = float(torch.linalg.norm(Xb))
    assert float(torch.linalg.norm(Xb - Xf)) / scale < 1e-5


def test_fp8_needs_byte_rows(gb):
    Y = W.gaussian_dominant(500, 20, 3, seed=1, dtype=np.float32)
    with pytest.raises(gb.MdsError) as e:
        gb.mds_interpolate(dev(Y), dev(W.landmarks(500, 100, seed=1)), 3, "fp8")
    assert e.value.status == 7


def test_image_fp8_full_size_sampled(gb):
    """The image-like configuration at full size (814,255 x 784 bytes, l = 2000,
    r = 10, FP8 nibble planes): sampled rows against the oracle's landmark MDS
    and Eq. (2)."""
    w = W.IMAGE_FP8
    Y = W.make_data(w, seed=0)
    idx = W.landmarks(w.n, w.l, seed=0)
    X, var, _ = gb.mds_interpolate(dev(Y), dev(idx), w.r, "fp8")
    X = host(X)
    L = Y[idx].astype(np.float64)
    D1 = O.sq_dist(L, L)
    X1, lam, _, _ = O.classical_mds(D1, w.r)
    rows = np.random.default_rng(0).choice(np.setdiff1d(np.arange(w.n), idx), 3000, replace=False)
    Xs = O.gower_interpolate(X1, lam, D1, O.sq_dist(Y[rows].astype(np.float64), L))
    both = np.concatenate([X[idx], X[rows]])
    ref = np.concatenate([X1, Xs])
    assert O.aligned_rel_error(both, ref) < TOL["bf16"]
    assert rel(host(var), lam / w.l) < LAM_TOL["f32"]


# ------------------------------------------------------ divide-and-conquer plans


def test_dc_plan_autotuned_graph(gb):
    """The plan's autotuned, graph-replayed run equals a direct call with the
    cluster size it chose, bit for bit, and the oracle within tolerance; a
    changed output buffer is captured again."""
    from paper_2007_11919_gb300.mds import DcPlan
    Y = W.gaussian_dominant(12_000, 100, 5, seed=4, dtype=np.float32)
    part = W.partitions_uneven(12_000, 20, 800, 1200, seed=4)
    Yd, anc, own = dev(Y), dev(part.anchors), dev(part.own)
    plan = DcPlan(12_000, 100, torch.float32, part.ptr, 20, 10, "f32", tune=True)
    X1, v1 = plan.execute(Yd, anc, own)
    info = plan.info()
    assert 1 <= info["cluster"] <= 16 and info["graph_nodes"] >= 8 and len(info["trial_ms"]) >= 2
    X2, v2 = plan.execute(Yd, anc, own)                       # graph replay, same buffers
    assert torch.equal(X1, X2) and torch.equal(v1, v2)
    Xd, vd = gb.mds_divide_conquer(Yd, anc, part.ptr, own, 10, "f32", cluster=info["cluster"])
    assert torch.equal(X2, Xd) and torch.equal(v2, vd)
    X3 = torch.zeros_like(X1)
    plan.execute(Yd, anc, own, X=X3)                          # new buffer: captured again
    assert torch.equal(X3, Xd)
    Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 10)
    assert O.aligned_rel_error(host(X2), Xo) < TOL["f32"]
    plan.close()


def test_tune_cache_round_trip(gb, tmp_path):
    """A tuning plan stores its measured cluster size in the cache file; a
    value stored under the same batch shape is then used, without timing, by
    a new tuning plan and by direct calls (whose results equal those of an
    explicit cluster size bit for bit)."""
    import json
    from paper_2007_11919_gb300 import mds as M
    path = tmp_path / "tune.json"
    M.mds_set_tune_cache(str(path))
    try:
        Y = W.gaussian_dominant(6000, 20, 4, seed=8, dtype=np.float32)
        part = W.partitions_uneven(6000, 12, 500, 700, seed=8)
        Yd, anc, own = dev(Y), dev(part.anchors), dev(part.own)
        plan = M.DcPlan(6000, 20, torch.float32, part.ptr, 12, 4, "f32", tune=True)
        plan.execute(Yd, anc, own)
        chosen = plan.info()["cluster"]
        plan.close()
        entries = json.loads(path.read_text())["entries"]
        assert len(entries) == 1 and entries[0]["value"] == chosen
        key = entries[0]["key"]
        assert key.startswith("k_lanczos") and "r=4" in key and "q=f32" in key
        assert M.mds_tune_cache_lookup(key) == chosen
        other = 3 if chosen != 3 else 2
        M.mds_tune_cache_store(key, other)
        plan = M.DcPlan(6000, 20, torch.float32, part.ptr, 12, 4, "f32", tune=True)
        X1, v1 = plan.execute(Yd, anc, own)
        info = plan.info()
        assert info["cluster"] == other and not any(info["trial_ms"])   # taken from the cache, nothing timed
        plan.close()
        X2, v2 = gb.mds_divide_conquer(Yd, anc, part.ptr, own, 4, "f32")
        Xe, ve = gb.mds_divide_conquer(Yd, anc, part.ptr, own, 4, "f32", cluster=other)
        assert torch.equal(X1, Xe) and torch.equal(X2, Xe) and torch.equal(v2, ve)
    finally:
        M.mds_set_tune_cache(None)
    assert M.mds_tune_cache_lookup("k_lanczos anything") == 0


def test_dc_plan_fixed_cluster_f64(gb):
    from paper_2007_11919_gb300.mds import DcPlan
    Y = W.gaussian_dominant(3000, 10, 3, seed=3)
    part = W.partitions_uneven(3000, 10, 300, 420, seed=3)
    plan = DcPlan(3000, 10, torch.float64, part.ptr, 10, 3, "f64", tune=False, cluster=3)
    X, var = plan.execute(dev(Y), dev(part.anchors), dev(part.own))
    assert plan.info()["cluster"] == 3
    Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 3)
    assert O.aligned_rel_error(host(X), Xo) < TOL["f64"]
    assert rel(host(var), lo) < LAM_TOL["f64"]


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
@pytest.mark.parametrize("n,d,c,lo,hi", [(6000, 784, 50, 900, 1100), (3000, 37, 12, 300, 420)])
def test_dc_u8_tensor_core_gram(gb, prec, n, d, c, lo, hi):
    """Divide-and-conquer of byte rows with the part Gram on tcgen05 (exact
    BF16 or E4M3 nibble operands): against the oracle, and against the FP32
    distance-tile path on the same data."""
    Y = W.image_like(n, d, seed=d)
    part = W.partitions_uneven(n, c, lo, hi, seed=d)
    r = 10 if d > 100 else 4
    X, var = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), r, prec)
    Xf, vf = gb.mds_divide_conquer(dev(Y), dev(part.anchors), part.ptr, dev(part.own), r, "f32")
    assert O.aligned_rel_error(host(X), host(Xf)) < 1e-5
    Xo, lo_, _ = O.divide_conquer_mds(Y.astype(np.float64), part.anchors, part.ptr, part.own, r)
    assert O.aligned_rel_error(host(X), Xo) < TOL["bf16"]
    assert rel(host(var), lo_) < LAM_TOL["f32"]


def test_dc_plan_execute_host_equals_device(gb):
    """A plan run on host buffers (pinned or pageable) gives the device run's
    result bitwise; the second host call replays the graph on the plan's own
    device buffers."""
    from paper_2007_11919_gb300.mds import DcPlan
    Y = W.gaussian_dominant(8000, 50, 5, seed=12, dtype=np.float32)
    part = W.partitions_uneven(8000, 20, 700, 1000, seed=12)
    plan = DcPlan(8000, 50, torch.float32, part.ptr, 20, 10, "f32", tune=False, cluster=4)
    Xd, vd = plan.execute(dev(Y), dev(part.anchors), dev(part.own))
    Yh = torch.from_numpy(Y).pin_memory()
    Xh, vh = plan.execute_host(Yh, torch.from_numpy(part.anchors), torch.from_numpy(part.own))
    assert not Xh.is_cuda and torch.equal(Xh, Xd.cpu()) and torch.equal(vh, vd.cpu())
    Xh2, vh2 = plan.execute_host(torch.from_numpy(Y), part.anchors, part.own)
    assert torch.equal(Xh2, Xd.cpu()) and torch.equal(vh2, vd.cpu())
    plan.close()


@pytest.fixture(scope="module")
def image_dc_case():
    """The image-like divide-and-conquer layout at its real part size: parts
    of 2,000 points (50 connecting points + 1,950 own), eight parts of which
    the last holds 1,050, d = 784 byte pixels, r = 10.  The oracle's parts
    (independent classical-MDS problems) are solved in a spawn pool."""
    n = 50 + 7 * 1950 + 1000
    part = W.partitions_equal(n, 2000, 50, seed=7)
    assert part.p == 8 and part.sizes()[-1] == 1050
    Y = W.image_like(n, 784, seed=7)
    with multiprocessing.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        Xo, lo, _ = O.divide_conquer_mds(Y, part.anchors, part.ptr, part.own, 10, map_fn=pool.map)
    return Y, part, Xo, lo


@pytest.mark.parametrize("prec", ["fp8", "bf16"])
def test_dc_image_parts_of_2000(gb, image_dc_case, prec):
    """Divide-and-conquer of image-like byte rows at the part layout of the
    full image-like workload (2,000-point parts, whole-row eigen-solver
    matvec): every row against the oracle after alignment, lambda-bar at
    1e-6; the autotuned graph plan gives the direct call's result bitwise."""
    from paper_2007_11919_gb300.mds import DcPlan
    Y, part, Xo, lo = image_dc_case
    Yd, anc, own = dev(Y), dev(part.anchors), dev(part.own)
    X, var = gb.mds_divide_conquer(Yd, anc, part.ptr, own, 10, prec)
    assert O.aligned_rel_error(host(X), Xo) < TOL["bf16"]
    assert rel(host(var), lo) < LAM_TOL["bf16"]
    plan = DcPlan(Y.shape[0], 784, torch.uint8, part.ptr, 50, 10, prec, tune=True)
    Xp, vp = plan.execute(Yd, anc, own)
    Xc, vc = gb.mds_divide_conquer(Yd, anc, part.ptr, own, 10, prec, cluster=plan.info()["cluster"])
    assert torch.equal(Xp, Xc) and torch.equal(vp, vc)
    assert O.aligned_rel_error(host(Xp), Xo) < TOL["bf16"]
    plan.close()


def test_dc_plan_fp8(gb):
    from paper_2007_11919_gb300.mds import DcPlan
    Y = W.image_like(5000, 784, seed=2)
    part = W.partitions_equal(5000, 1000, 50, seed=2)
    plan = DcPlan(5000, 784, torch.uint8, part.ptr, 50, 10, "fp8", tune=True)
    Yd, anc, own = dev(Y), dev(part.anchors), dev(part.own)
    X, var = plan.execute(Yd, anc, own)
    Xd, vd = gb.mds_divide_conquer(Yd, anc, part.ptr, own, 10, "fp8", cluster=plan.info()["cluster"])
    assert torch.equal(X, Xd) and torch.equal(var, vd)
    Xo, lo_, _ = O.divide_conquer_mds(Y.astype(np.float64), part.anchors, part.ptr, part.own, 10)
    assert O.aligned_rel_error(host(X), Xo) < TOL["bf16"]


# ------------------------------------------------ interpolation from host memory

@pytest.mark.parametrize("prec,kind", [("bf16", "f32"), ("f32", "f32"), ("f64", "f64"), ("f32", "f64"),
                                       ("fp8", "u8"), ("bf16", "u8")])
@pytest.mark.parametrize("n,d,l,r,chunk", [(5000, 100, 300, 10, 1024), (2999, 37, 129, 3, 700),
                                           (700, 20, 300, 5, 0)])
def test_interp_host_equals_device(gb, prec, kind, n, d, l, r, chunk):
    """mds_interpolate_host (host rows, chunked copies overlapping the landmark
    eigenproblem and the projection) gives bitwise the result of
    mds_interpolate on a device copy: same X (landmark rows included), same
    variances, and a model that embeds identically; ragged last chunk, chunks
    smaller than a tile, one chunk for all rows."""
    if kind == "u8":
        d = 784 if d == 100 else d
        Y = W.image_like(n, d, seed=n + d)
    else:
        Y = W.gaussian_dominant(n, d, min(5, d), seed=n + d, dtype=np.float64 if kind == "f64" else np.float32)
    idx = W.landmarks(n, l, seed=n + l)
    Xd, vd, md = gb.mds_interpolate(dev(Y), dev(idx), r, prec, want_model=True)
    Yh = torch.from_numpy(np.ascontiguousarray(Y)).pin_memory()
    Xh, vh, mh = gb.mds_interpolate_host(Yh, torch.from_numpy(idx), r, prec, want_model=True, chunk_rows=chunk)
    assert not Xh.is_cuda and Xh.shape == (n, r)
    assert torch.equal(Xh, Xd.cpu())
    assert torch.equal(vh, vd.cpu())
    probe = dev(Y[:257])
    assert torch.equal(gb.mds_embed_new(mh, probe), gb.mds_embed_new(md, probe))


def test_interp_host_pageable_and_errors(gb):
    """Pageable host rows give the same result (the copies just do not
    overlap); a landmark index outside [0, n) is an argument error."""
    n, d, l, r = 3000, 50, 200, 4
    Y = W.gaussian_dominant(n, d, 5, seed=3, dtype=np.float32)
    idx = W.landmarks(n, l, seed=4)
    Xd, vd, _ = gb.mds_interpolate(dev(Y), dev(idx), r, "bf16")
    Xh, vh, _ = gb.mds_interpolate_host(torch.from_numpy(Y), torch.from_numpy(idx), r, "bf16", chunk_rows=512)
    assert torch.equal(Xh, Xd.cpu()) and torch.equal(vh, vd.cpu())
    bad = idx.copy()
    bad[3] = n
    with pytest.raises(gb.MdsError):
        gb.mds_interpolate_host(torch.from_numpy(Y), torch.from_numpy(bad), r, "bf16")
    with pytest.raises(ValueError):
        gb.mds_interpolate_host(dev(Y), torch.from_numpy(idx), r, "bf16")
