"""The C-ABI library builds, loads and exports every entry point declared in
include/gbmds.h; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbmds.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2007_11919_gb300 import build
    path = build.build()
    from paper_2007_11919_gb300.mds import _lib
    assert os.path.samefile(path, os.path.join(ROOT, "paper_2007_11919_gb300", "libgbmds.so"))
    return _lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mds_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("mds_classical", "mds_interpolate", "mds_divide_conquer", "mds_embed_new"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"


def test_status_strings(lib):
    assert lib.mds_version() == 1
    for s in range(10):
        assert lib.mds_status_str(s)
    assert lib.mds_status_str(4) == b"fewer than r positive eigenvalues"


def _opts(**kw):
    from paper_2007_11919_gb300.mds import MdsOpts
    return MdsOpts(**kw)


def test_argument_checks_without_gpu(lib):
    o = _opts(prec=1)
    p = ctypes.c_void_p(8)
    # null data / bad sizes / bad r are rejected before any CUDA call
    assert lib.mds_classical(None, 1, 100, 3, 2, ctypes.byref(o), p, p) == 1
    assert lib.mds_classical(p, 1, 100, 3, 100, ctypes.byref(o), p, p) == 1
    assert lib.mds_classical(p, 7, 100, 3, 2, ctypes.byref(o), p, p) == 1
    assert lib.mds_interpolate(p, 1, 100, 3, p, 200, 2, ctypes.byref(o), p, p, None) == 1
    assert lib.mds_interpolate(p, 1, 100, 3, p, 50, 40, ctypes.byref(o), p, p, None) == 1
    bad = _opts(prec=9)
    assert lib.mds_classical(p, 1, 100, 3, 2, ctypes.byref(bad), p, p) == 1
    flags = _opts(prec=1, flags=2)   # an unknown flag bit
    assert lib.mds_classical(p, 1, 100, 3, 2, ctypes.byref(flags), p, p) == 1
    # divide-and-conquer: c must exceed r (Procrustes needs c >= r + 1)
    ptr = np.array([0, 100, 200], dtype=np.int64)
    pp = ptr.ctypes.data_as(ctypes.c_void_p)
    assert lib.mds_divide_conquer(p, 1, 220, 3, 2, pp, p, p, 3, 3, ctypes.byref(o), p, p) == 1
    ptr_bad = np.array([5, 100, 200], dtype=np.int64)
    assert lib.mds_divide_conquer(p, 1, 220, 3, 2, ptr_bad.ctypes.data_as(ctypes.c_void_p), p, p, 10, 3,
                                  ctypes.byref(o), p, p) == 1
    # missing workspace is reported as such (still no GPU work)
    assert lib.mds_classical(p, 1, 100, 3, 2, ctypes.byref(o), p, p) == 8
    # MDS_FLAG_FULL_MATVEC is a known flag: the same call gets as far as the workspace check
    full = _opts(prec=1, flags=1)
    assert lib.mds_classical(p, 1, 100, 3, 2, ctypes.byref(full), p, p) == 8
    # FP8 needs uint8 data paths not built for classical MDS
    o8 = _opts(prec=3)
    assert lib.mds_classical(p, 2, 100, 3, 2, ctypes.byref(o8), p, p) == 7


def test_workspace_sizes(lib):
    s_small = lib.mds_classical_workspace_size(100, 3, 2, 1)
    s_big = lib.mds_classical_workspace_size(1000, 3, 2, 1)
    assert 0 < s_small < s_big
    assert lib.mds_classical_workspace_size(0, 3, 2, 1) == 0
    # Q (n x n FP64) dominates the classical workspace
    assert s_big >= 1000 * 1000 * 8
    ptr = np.array([0] + list(np.cumsum([1000] * 10)), dtype=np.int64)
    w = lib.mds_divide_conquer_workspace_size(10_020, 100, 10, ptr.ctypes.data_as(ctypes.c_void_p), 20, 10, 1)
    assert w >= 10 * 1020 * 1020 * 8
    assert lib.mds_interpolate_workspace_size(10_000, 100, 500, 10, 2) > lib.mds_interpolate_workspace_size(
        10_000, 100, 500, 10, 1)


def test_host_interpolation_checks_without_gpu(lib):
    """mds_interpolate_host checks its host-side arguments (landmark range,
    chunk size, workspace) before any CUDA work."""
    o = _opts(prec=1)
    p = ctypes.c_void_p(8)
    good = np.arange(0, 200, 2, dtype=np.int64)            # 100 landmarks of 1,000 rows
    bad = good.copy()
    bad[7] = 1000                                           # outside [0, n)
    neg = good.copy()
    neg[0] = -1
    gp, bp, np_ = (a.ctypes.data_as(ctypes.c_void_p) for a in (good, bad, neg))
    assert lib.mds_interpolate_host(p, 1, 1000, 8, bp, 100, 3, 0, ctypes.byref(o), p, p, None) == 1
    assert lib.mds_interpolate_host(p, 1, 1000, 8, np_, 100, 3, 0, ctypes.byref(o), p, p, None) == 1
    assert lib.mds_interpolate_host(p, 1, 1000, 8, gp, 100, 3, -5, ctypes.byref(o), p, p, None) == 1
    assert lib.mds_interpolate_host(p, 1, 1000, 8, gp, 100, 100, 0, ctypes.byref(o), p, p, None) == 1
    # valid arguments, no workspace: reported before anything touches the data
    assert lib.mds_interpolate_host(p, 1, 1000, 8, gp, 100, 3, 0, ctypes.byref(o), p, p, None) == 8
    # the host variant's workspace holds a device copy of Y and X on top
    dev = lib.mds_interpolate_workspace_size(10_000, 100, 500, 10, 2)
    host = lib.mds_interpolate_host_workspace_size(10_000, 100, 500, 10, 2, 1)
    assert host >= dev + 10_000 * 100 * 4 + 10_000 * 10 * 4
    assert lib.mds_interpolate_host_workspace_size(10_000, 100, 500, 10, 2, 9) == 0


def test_affine_interpolation_checks_without_gpu(lib):
    o = _opts(prec=1)
    p = ctypes.c_void_p(8)
    assert lib.mds_interpolate_affine(None, 1, 1000, 8, p, 100, 3, ctypes.byref(o), p, p) == 1
    assert lib.mds_interpolate_affine(p, 1, 1000, 8, p, 2000, 3, ctypes.byref(o), p, p) == 1   # l > n
    assert lib.mds_interpolate_affine(p, 1, 1000, 8, p, 100, 100, ctypes.byref(o), p, p) == 1  # r >= l
    ob = _opts(prec=2)
    assert lib.mds_interpolate_affine(p, 1, 1000, 8, p, 100, 3, ctypes.byref(ob), p, p) == 7   # BF16
    assert lib.mds_interpolate_affine(p, 1, 1000, 8, p, 100, 3, ctypes.byref(o), p, p) == 8    # no workspace
    assert lib.mds_interpolate_affine_workspace_size(1000, 8, 100, 3, 2) == 0
    small = lib.mds_interpolate_affine_workspace_size(1000, 8, 100, 3, 1)
    assert small > 100 * 100 * 4 and small < lib.mds_interpolate_affine_workspace_size(1000, 8, 400, 3, 1)


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2007_11919_gb300.mds as M
    monkeypatch.setattr(M, "_L", None)
    monkeypatch.setattr(M, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        M._lib()


def test_server_argument_checks_without_gpu(lib):
    from paper_2007_11919_gb300.mds import MdsServerOpts, _server_lib
    L = _server_lib()
    o = MdsServerOpts(slots=4, flags=0, slot_bytes=0, max_batch_rows=0)
    h = ctypes.c_void_p()
    assert L.mds_server_create(None, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    arr = (ctypes.c_void_p * 1)(None)
    assert L.mds_server_create(arr, 1, ctypes.byref(o), ctypes.byref(h)) == 1   # null model
    bad = MdsServerOpts(slots=99, flags=0, slot_bytes=0, max_batch_rows=0)
    assert L.mds_server_create(arr, 1, ctypes.byref(bad), ctypes.byref(h)) == 1
    t = ctypes.c_uint64()
    p = ctypes.c_void_p(8)
    assert L.mds_server_submit(None, 0, p, 1, 10, p, ctypes.byref(t)) == 1
    st = ctypes.c_int()
    assert L.mds_server_wait(None, 1, 1.0, ctypes.byref(st), None) == 1
    assert L.mds_server_destroy(None) == 1


def test_dc_plan_argument_checks_without_gpu(lib):
    from paper_2007_11919_gb300.mds import MdsOpts
    lib.mds_dc_plan_create.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.mds_dc_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    o = MdsOpts(prec=1)
    ptr = np.array([0, 100, 200], dtype=np.int64)
    pp = ptr.ctypes.data_as(ctypes.c_void_p)
    # c must exceed r; the plan owns its workspace; BF16 / FP8 D&C not built
    assert lib.mds_dc_plan_create(220, 3, 1, 2, pp, 3, 3, ctypes.byref(o), 1, ctypes.byref(h)) == 1
    ow = MdsOpts(prec=1, workspace=ctypes.c_void_p(256), workspace_bytes=1024)
    assert lib.mds_dc_plan_create(220, 3, 1, 2, pp, 10, 3, ctypes.byref(ow), 1, ctypes.byref(h)) == 1
    ob = MdsOpts(prec=2)
    assert lib.mds_dc_plan_create(220, 3, 1, 2, pp, 10, 3, ctypes.byref(ob), 1, ctypes.byref(h)) == 7
    assert lib.mds_dc_plan_create(220, 3, 1, 2, pp, 10, 3, ctypes.byref(o), 1, None) == 1


def test_maxmin_argument_checks_without_gpu(lib):
    o = _opts(prec=0)
    p = ctypes.c_void_p(8)
    lib.mds_landmarks_maxmin.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    lib.mds_landmarks_maxmin.restype = ctypes.c_int
    assert lib.mds_landmarks_maxmin(p, 1, 100, 4, 0, 0, ctypes.byref(o), p) == 1      # l < 1
    assert lib.mds_landmarks_maxmin(p, 1, 100, 4, 101, 0, ctypes.byref(o), p) == 1    # l > n
    assert lib.mds_landmarks_maxmin(p, 1, 100, 4, 10, 100, ctypes.byref(o), p) == 1   # first out of range
    assert lib.mds_landmarks_maxmin(None, 1, 100, 4, 10, 0, ctypes.byref(o), p) == 1
    assert lib.mds_landmarks_maxmin(p, 1, 100, 20000, 10, 0, ctypes.byref(o), p) == 7  # rows too wide
    assert lib.mds_landmarks_maxmin(p, 1, 100, 4, 10, 0, ctypes.byref(o), p) == 8     # no workspace


def test_fast_tree_checks_without_gpu(lib):
    """The division tree of fast MDS is validated on the host: a well-formed
    tree gets a workspace size, malformed ones get 0 (and MDS_ERR_ARG from
    mds_fast before any device work)."""
    import workloads as W
    lib.mds_fast_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.mds_fast_workspace_size.restype = ctypes.c_size_t
    lib.mds_fast.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p]
    lib.mds_fast.restype = ctypes.c_int
    tree = W.fast_mds_tree(5000, 400, 20, seed=2)
    _, rg, par = W.flatten_fast_tree(tree)

    def size(rg_, par_, s=20, r=3):
        rg_ = np.ascontiguousarray(rg_, dtype=np.int64)
        par_ = np.ascontiguousarray(par_, dtype=np.int32)
        return lib.mds_fast_workspace_size(5000, 8, len(par_), rg_.ctypes.data, par_.ctypes.data, s, r, 1)

    assert size(rg, par) > 0
    bad = rg.copy()
    bad[3, 0] += 1                      # a gap between two children
    assert size(bad, par) == 0
    bad = par.copy()
    bad[4] = 4                          # a node that is its own parent
    assert size(rg, bad) == 0
    bad = par.copy()
    bad[0] = 0                          # no root
    assert size(rg, bad) == 0
    assert size(rg, par, s=3, r=3) == 0            # s < r + 1
    assert size(rg, par, s=300) == 0               # subsets smaller than s
    assert size(np.array([[0, 5000]]), np.array([-1])) > 0         # one leaf: classical MDS
    assert lib.mds_fast_workspace_size(20000, 8, 1, np.array([0, 20000], dtype=np.int64).ctypes.data,
                                       np.array([-1], dtype=np.int32).ctypes.data, 20, 3, 1) == 0  # leaf too big


def test_pivot_argument_checks_without_gpu(lib):
    """Pivot MDS: argument errors, unsupported precisions and row widths
    beyond the scatter kernel's staging (d > 4096) answer on the host."""
    o = _opts(prec=1)
    p = ctypes.c_void_p(8)
    lib.mds_pivot_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.mds_pivot_workspace_size.restype = ctypes.c_size_t
    lib.mds_pivot.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mds_pivot.restype = ctypes.c_int
    assert lib.mds_pivot_workspace_size(100000, 100, 1000, 10, 1) > 100 * 100 * 8
    assert lib.mds_pivot_workspace_size(100000, 4096, 1000, 10, 1) > 0
    assert lib.mds_pivot_workspace_size(100000, 4097, 1000, 10, 1) == 0
    assert lib.mds_pivot_workspace_size(100000, 100, 1000, 10, 2) == 0          # BF16
    assert lib.mds_pivot(None, 1, 1000, 8, p, 100, 3, ctypes.byref(o), p, p) == 1
    assert lib.mds_pivot(p, 1, 1000, 8, p, 100, 9, ctypes.byref(o), p, p) == 1    # r > d
    assert lib.mds_pivot(p, 1, 1000, 8, p, 2000, 3, ctypes.byref(o), p, p) == 1   # l > n
    assert lib.mds_pivot(p, 1, 1000, 4097, p, 100, 3, ctypes.byref(o), p, p) == 7
    assert lib.mds_pivot(p, 1, 1000, 8, p, 100, 3, ctypes.byref(_opts(prec=2)), p, p) == 7
    assert lib.mds_pivot(p, 1, 1000, 8, p, 100, 3, ctypes.byref(o), p, p) == 8    # no workspace


def test_tune_cache_file_without_gpu(lib, tmp_path):
    """The tuning cache: absent keys read 0, stores add and replace entries in
    a JSON file, malformed keys and a cache that is off are refused."""
    import json
    from paper_2007_11919_gb300 import mds as M
    path = tmp_path / "tune.json"
    assert M.mds_tune_cache_lookup("k_lanczos cluster p=1") == 0          # cache off
    with pytest.raises(M.MdsError):
        M.mds_tune_cache_store("k_lanczos cluster p=1", 4)
    M.mds_set_tune_cache(str(path))
    try:
        assert M.mds_tune_cache_lookup("k_lanczos cluster p=1") == 0
        M.mds_tune_cache_store("k_lanczos cluster p=1", 4)
        M.mds_tune_cache_store("k_lanczos cluster p=2", 7)
        M.mds_tune_cache_store("k_lanczos cluster p=1", 5)                # replaces
        doc = json.loads(path.read_text())
        assert doc["gbmds_tune_cache"] == 1
        assert {e["key"]: e["value"] for e in doc["entries"]} == {"k_lanczos cluster p=1": 5,
                                                                  "k_lanczos cluster p=2": 7}
        assert M.mds_tune_cache_lookup("k_lanczos cluster p=2") == 7
        for bad in ['a"b', "a\\b", "a\nb", "", "x" * 1025]:
            with pytest.raises(M.MdsError):
                M.mds_tune_cache_store(bad, 1)
        assert not any(p.name.startswith("tune.json.tmp") for p in tmp_path.iterdir())
    finally:
        M.mds_set_tune_cache(None)
