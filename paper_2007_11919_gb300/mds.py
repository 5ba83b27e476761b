"""Python binding of libgbmds.so (argument marshalling only).

Every function here has the name of the C entry point it calls (see
include/gbmds.h): it checks tensor placement and dtypes, allocates the output
tensors and the scratch workspace with PyTorch on the data's device, passes
raw pointers and the current CUDA stream, and turns a non-zero status into
``MdsError``.  All arithmetic happens in the CUDA kernels behind the C ABI;
there is no CPU fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbmds.so")

PREC = {"f64": 0, "f32": 1, "bf16": 2, "fp8": 3}
FLAG_FULL_MATVEC = 1   # mds_opts.flags: stream every row of Q whole (no symmetric ranges)
DTYPE = {torch.float64: 0, torch.float32: 1, torch.uint8: 2}
STATUS = {0: "MDS_OK", 1: "MDS_ERR_ARG", 2: "MDS_ERR_NOMEM", 3: "MDS_ERR_CUDA", 4: "MDS_ERR_RANK",
          5: "MDS_ERR_NOCONV", 6: "MDS_ERR_TIMEOUT", 7: "MDS_ERR_UNSUPPORTED",
          8: "MDS_ERR_WORKSPACE", 9: "MDS_ERR_IO"}


class MdsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_lib().mds_status_str(status).decode()})")


class MdsOpts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("eig_tol", ctypes.c_double), ("rank_tol", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("cluster", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


_L = None
_P, _I, _I32, _I64, _D, _SZ = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_double, ctypes.c_size_t)


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_2007_11919_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "mds_status_str": (ctypes.c_char_p, [_I]),
            "mds_version": (_I, []),
            "mds_classical_workspace_size": (_SZ, [_I64, _I, _I, _I]),
            "mds_classical": (_I, [_P, _I, _I64, _I, _I, _P, _P, _P]),
            "mds_classical_dist_workspace_size": (_SZ, [_I64, _I]),
            "mds_classical_dist": (_I, [_P, _I64, _I, _P, _P, _P]),
            "mds_interpolate_workspace_size": (_SZ, [_I64, _I, _I, _I, _I]),
            "mds_interpolate": (_I, [_P, _I, _I64, _I, _P, _I, _I, _P, _P, _P, _P]),
            "mds_interpolate_affine_workspace_size": (_SZ, [_I64, _I, _I, _I, _I]),
            "mds_interpolate_affine": (_I, [_P, _I, _I64, _I, _P, _I, _I, _P, _P, _P]),
            "mds_interpolate_host_workspace_size": (_SZ, [_I64, _I, _I, _I, _I, _I]),
            "mds_interpolate_host": (_I, [_P, _I, _I64, _I, _P, _I, _I, _I64, _P, _P, _P, _P]),
            "mds_embed_new_workspace_size": (_SZ, [_P, _I64]),
            "mds_embed_new": (_I, [_P, _P, _I, _I64, _P, _P]),
            "mds_model_info": (_I, [_P, _P, _P, _P, _P, _P]),
            "mds_model_save": (_I, [_P, ctypes.c_char_p]),
            "mds_model_load": (_I, [ctypes.c_char_p, _P]),
            "mds_model_free": (None, [_P]),
            "mds_pivot_workspace_size": (_SZ, [_I64, _I, _I, _I, _I]),
            "mds_pivot": (_I, [_P, _I, _I64, _I, _P, _I, _I, _P, _P, _P]),
            "mds_fast_workspace_size": (_SZ, [_I64, _I, _I, _P, _P, _I, _I, _I]),
            "mds_fast": (_I, [_P, _I, _I64, _I, _P, _I, _P, _P, _I, _I, _P, _P, _P]),
            "mds_landmarks_maxmin_workspace_size": (_SZ, [_I64, _I]),
            "mds_landmarks_maxmin": (_I, [_P, _I, _I64, _I, _I, _I64, _P, _P]),
            "mds_divide_conquer_workspace_size": (_SZ, [_I64, _I, _I, _P, _I, _I, _I]),
            "mds_divide_conquer": (_I, [_P, _I, _I64, _I, _I, _P, _P, _P, _I, _I, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check(status: int, where: str):
    if status != 0:
        raise MdsError(status, where)


def _opts(device, prec, nbytes, stream=None, max_steps=0, eig_tol=0.0, rank_tol=0.0, cluster=0,
          workspace=None, full_matvec=False):
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
    st = stream if stream is not None else torch.cuda.current_stream(device)
    o = MdsOpts(prec=PREC[prec], max_steps=max_steps, eig_tol=eig_tol, rank_tol=rank_tol,
                stream=ctypes.c_void_p(st.cuda_stream), workspace=_ptr(workspace),
                workspace_bytes=workspace.numel(), cluster=cluster,
                flags=FLAG_FULL_MATVEC if full_matvec else 0)
    return o, workspace


def _data(Y):
    if not (isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dim() == 2 and Y.is_contiguous()):
        raise ValueError("data must be a contiguous 2-D CUDA tensor")
    if Y.dtype not in DTYPE:
        raise ValueError(f"unsupported dtype {Y.dtype}")
    return DTYPE[Y.dtype]


def _idx(t, device):
    t = torch.as_tensor(t, dtype=torch.int64)
    return t.to(device).contiguous()


def _xdtype(prec):
    return torch.float64 if prec == "f64" else torch.float32


def mds_version() -> int:
    return _lib().mds_version()


def mds_classical(Y, r, prec="f64", **kw):
    """Classical MDS of the rows of Y (Section 2). Returns (X n x r, lambda r)."""
    dt = _data(Y)
    n, d = Y.shape
    L = _lib()
    o, ws = _opts(Y.device, prec, L.mds_classical_workspace_size(n, d, r, PREC[prec]), **kw)
    X = torch.empty((n, r), dtype=_xdtype(prec), device=Y.device)
    lam = torch.empty(r, dtype=torch.float64, device=Y.device)
    _check(L.mds_classical(_ptr(Y), dt, n, d, r, ctypes.byref(o), _ptr(X), _ptr(lam)), "mds_classical")
    return X, lam


def mds_classical_dist(D2, r, **kw):
    """Classical MDS of an n x n squared-distance matrix (FP64, on the GPU)."""
    if not (D2.is_cuda and D2.dtype == torch.float64 and D2.is_contiguous() and D2.dim() == 2):
        raise ValueError("D2 must be a contiguous n x n float64 CUDA tensor")
    n = D2.shape[0]
    L = _lib()
    o, ws = _opts(D2.device, "f64", L.mds_classical_dist_workspace_size(n, r), **kw)
    X = torch.empty((n, r), dtype=torch.float64, device=D2.device)
    lam = torch.empty(r, dtype=torch.float64, device=D2.device)
    _check(L.mds_classical_dist(_ptr(D2), n, r, ctypes.byref(o), _ptr(X), _ptr(lam)), "mds_classical_dist")
    return X, lam


class Model:
    """Owner of an mds_model handle (device-resident landmark configuration)."""

    def __init__(self, handle: int, device):
        self.handle = ctypes.c_void_p(handle)
        self.device = torch.device(device)

    def info(self):
        l, d, r, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib().mds_model_info(self.handle, ctypes.byref(l), ctypes.byref(d), ctypes.byref(r),
                                     ctypes.byref(p), None), "mds_model_info")
        lam = (ctypes.c_double * r.value)()
        _check(_lib().mds_model_info(self.handle, None, None, None, None, lam), "mds_model_info")
        inv = {v: k for k, v in PREC.items()}
        return {"l": l.value, "d": d.value, "r": r.value, "prec": inv[p.value], "lambda": list(lam)}

    def save(self, path: str):
        _check(_lib().mds_model_save(self.handle, path.encode()), "mds_model_save")

    @classmethod
    def load(cls, path: str, device="cuda"):
        h = ctypes.c_void_p()
        with torch.cuda.device(torch.device(device)):
            _check(_lib().mds_model_load(path.encode(), ctypes.byref(h)), "mds_model_load")
        return cls(h.value, device)

    def free(self):
        if self.handle and self.handle.value:
            _lib().mds_model_free(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mds_interpolate(Y, landmark_idx, r, prec="f32", want_model=False, **kw):
    """Interpolation MDS (Section 3.1). Returns (X n x r, var r, Model or None)."""
    dt = _data(Y)
    n, d = Y.shape
    idx = _idx(landmark_idx, Y.device)
    l = idx.numel()
    L = _lib()
    o, ws = _opts(Y.device, prec, L.mds_interpolate_workspace_size(n, d, l, r, PREC[prec]), **kw)
    X = torch.empty((n, r), dtype=_xdtype(prec), device=Y.device)
    var = torch.empty(r, dtype=torch.float64, device=Y.device)
    h = ctypes.c_void_p()
    _check(L.mds_interpolate(_ptr(Y), dt, n, d, _ptr(idx), l, r, ctypes.byref(o), _ptr(X), _ptr(var),
                             ctypes.byref(h) if want_model else None), "mds_interpolate")
    return X, var, (Model(h.value, Y.device) if want_model else None)


def mds_interpolate_affine(Y, landmark_idx, r, prec="f32", **kw):
    """Interpolation MDS (Section 3.1) in its affine form for coordinate rows:
    X = (Y - y_L) U_r with U_r the landmarks' principal axes scaled by
    Lambda^{-1/2} (Eq. (2) for Euclidean distances).  prec "f64" or "f32".
    Returns (X n x r, var r)."""
    dt = _data(Y)
    n, d = Y.shape
    idx = _idx(landmark_idx, Y.device)
    l = idx.numel()
    L = _lib()
    o, ws = _opts(Y.device, prec, L.mds_interpolate_affine_workspace_size(n, d, l, r, PREC[prec]), **kw)
    X = torch.empty((n, r), dtype=_xdtype(prec), device=Y.device)
    var = torch.empty(r, dtype=torch.float64, device=Y.device)
    _check(L.mds_interpolate_affine(_ptr(Y), dt, n, d, _ptr(idx), l, r, ctypes.byref(o), _ptr(X), _ptr(var)),
           "mds_interpolate_affine")
    return X, var


def mds_interpolate_host(Y, landmark_idx, r, prec="f32", want_model=False, chunk_rows=0, out=None,
                         device=None, **kw):
    """Interpolation MDS (Section 3.1) of host-resident rows: ``Y`` is a 2-D CPU
    tensor (pin it for the copies to overlap the computation), the result X and
    var are CPU tensors (X pinned unless ``out`` is given).  Bitwise equal to
    ``mds_interpolate`` on a device copy of ``Y``."""
    if not (isinstance(Y, torch.Tensor) and not Y.is_cuda and Y.dim() == 2 and Y.is_contiguous()):
        raise ValueError("data must be a contiguous 2-D CPU tensor")
    if Y.dtype not in DTYPE:
        raise ValueError(f"unsupported dtype {Y.dtype}")
    dt = DTYPE[Y.dtype]
    n, d = Y.shape
    idx = torch.as_tensor(landmark_idx, dtype=torch.int64).cpu().contiguous()
    l = idx.numel()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    L = _lib()
    o, ws = _opts(dev, prec, L.mds_interpolate_host_workspace_size(n, d, l, r, PREC[prec], dt), **kw)
    X = out if out is not None else torch.empty((n, r), dtype=_xdtype(prec), pin_memory=True)
    if X.is_cuda or X.shape != (n, r) or X.dtype != _xdtype(prec) or not X.is_contiguous():
        raise ValueError("out must be a contiguous CPU tensor of shape (n, r) and the result dtype")
    var = torch.empty(r, dtype=torch.float64)
    h = ctypes.c_void_p()
    _check(L.mds_interpolate_host(_ptr(Y), dt, n, d, _ptr(idx), l, r, int(chunk_rows), ctypes.byref(o), _ptr(X),
                                  _ptr(var), ctypes.byref(h) if want_model else None), "mds_interpolate_host")
    return X, var, (Model(h.value, dev) if want_model else None)


def mds_embed_new(model: Model, Ynew, prec=None, **kw):
    """Gower's formula (Eq. (2)) for new rows against a stored model."""
    dt = _data(Ynew)
    m = Ynew.shape[0]
    info_prec = prec if prec is not None else model.info()["prec"]
    r = model.info()["r"] if "r" not in kw else kw.pop("r")
    L = _lib()
    o, ws = _opts(Ynew.device, info_prec, L.mds_embed_new_workspace_size(model.handle, m), **kw)
    X = torch.empty((m, r), dtype=_xdtype(info_prec), device=Ynew.device)
    _check(L.mds_embed_new(model.handle, _ptr(Ynew), dt, m, ctypes.byref(o), _ptr(X)), "mds_embed_new")
    return X


def mds_pivot(Y, pivot_idx, r, prec="f32", **kw):
    """Pivot MDS (Section 3.1) of the rows of Y with the given pivot rows.
    Returns (X n x r, var r)."""
    dt = _data(Y)
    n, d = Y.shape
    idx = _idx(pivot_idx, Y.device)
    l = idx.numel()
    L = _lib()
    o, ws = _opts(Y.device, prec, L.mds_pivot_workspace_size(n, d, l, r, PREC[prec]), **kw)
    X = torch.empty((n, r), dtype=_xdtype(prec), device=Y.device)
    var = torch.empty(r, dtype=torch.float64, device=Y.device)
    _check(L.mds_pivot(_ptr(Y), dt, n, d, _ptr(idx), l, r, ctypes.byref(o), _ptr(X), _ptr(var)), "mds_pivot")
    return X, var


def mds_fast(Y, perm, node_range, node_parent, s, r, prec="f32", **kw):
    """Fast MDS (Section 3.3) over a given division tree: ``perm`` (rows in
    the division's order), ``node_range`` (nnodes x 2 host array of [begin,
    end) in perm) and ``node_parent`` (host, -1 for the root).  Returns
    (X n x r, var r)."""
    dt = _data(Y)
    n, d = Y.shape
    pm = _idx(perm, Y.device)
    rng = np.ascontiguousarray(np.asarray(node_range, dtype=np.int64).reshape(-1))
    par = np.ascontiguousarray(np.asarray(node_parent, dtype=np.int32))
    nn = len(par)
    rp, pp = rng.ctypes.data_as(ctypes.c_void_p), par.ctypes.data_as(ctypes.c_void_p)
    L = _lib()
    o, ws = _opts(Y.device, prec, L.mds_fast_workspace_size(n, d, nn, rp, pp, s, r, PREC[prec]), **kw)
    X = torch.empty((n, r), dtype=_xdtype(prec), device=Y.device)
    var = torch.empty(r, dtype=torch.float64, device=Y.device)
    _check(L.mds_fast(_ptr(Y), dt, n, d, _ptr(pm), nn, rp, pp, s, r, ctypes.byref(o), _ptr(X), _ptr(var)),
           "mds_fast")
    return X, var


def mds_landmarks_maxmin(Y, l, first=0, **kw):
    """LMDS's MaxMin choice of l landmarks (Section 3.1) starting from row
    ``first``; returns the l row indices (int64, on Y's device) in the order
    chosen, ready for ``mds_interpolate``."""
    dt = _data(Y)
    n, d = Y.shape
    L = _lib()
    o, ws = _opts(Y.device, "f64", L.mds_landmarks_maxmin_workspace_size(n, d), **kw)
    idx = torch.empty(l, dtype=torch.int64, device=Y.device)
    _check(L.mds_landmarks_maxmin(_ptr(Y), dt, n, d, l, int(first), ctypes.byref(o), _ptr(idx)),
           "mds_landmarks_maxmin")
    return idx


def mds_divide_conquer(Y, anchors, part_ptr, part_own, r, prec="f32", **kw):
    """Divide-and-conquer MDS (Section 3.2). ``part_ptr`` is host data (p+1
    offsets); ``anchors`` and ``part_own`` index rows of Y.  Returns (X, var)."""
    dt = _data(Y)
    n, d = Y.shape
    anc = _idx(anchors, Y.device)
    own = _idx(part_own, Y.device)
    ptr = np.ascontiguousarray(np.asarray(part_ptr, dtype=np.int64))
    p = len(ptr) - 1
    c = anc.numel()
    pp = ptr.ctypes.data_as(ctypes.c_void_p)
    L = _lib()
    o, ws = _opts(Y.device, prec, L.mds_divide_conquer_workspace_size(n, d, p, pp, c, r, PREC[prec]), **kw)
    X = torch.zeros((n, r), dtype=_xdtype(prec), device=Y.device)
    var = torch.empty(r, dtype=torch.float64, device=Y.device)
    _check(L.mds_divide_conquer(_ptr(Y), dt, n, d, p, pp, _ptr(own), _ptr(anc), c, r, ctypes.byref(o),
                                _ptr(X), _ptr(var)), "mds_divide_conquer")
    return X, var


class MdsStats(ctypes.Structure):
    _fields_ = [("stage_ms", ctypes.c_double * 5), ("launches", ctypes.c_int64),
                ("eig_steps", ctypes.c_int64), ("eig_flops", ctypes.c_double),
                ("eig_qbytes", ctypes.c_double), ("problems", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("eig_qread", ctypes.c_double)]


STAGES = ("prep", "dist", "center", "eig", "post")


def mds_set_timing(on: bool):
    """Record CUDA events between pipeline stages of later calls (this thread)."""
    L = _lib()
    L.mds_set_timing.argtypes = [_I]
    L.mds_set_timing.restype = None
    L.mds_set_timing(1 if on else 0)


def mds_last_stats() -> dict:
    """Stage times, launch count and eigen-solver work of the last call (this thread)."""
    L = _lib()
    L.mds_last_stats.argtypes = [_P]
    L.mds_last_stats.restype = _I
    s = MdsStats()
    _check(L.mds_last_stats(ctypes.byref(s)), "mds_last_stats")
    return {"stage_ms": dict(zip(STAGES, list(s.stage_ms))), "launches": s.launches,
            "eig_steps": s.eig_steps, "eig_flops": s.eig_flops, "eig_qbytes": s.eig_qbytes,
            "problems": s.problems, "cluster": s.cluster, "eig_qread": s.eig_qread}


def mds_set_wait_limit_ns(ns: int):
    """Failure injection: the team eigen-solver's grid-barrier waits give up
    after ``ns`` nanoseconds (0 = the default 2 s); process-wide."""
    L = _lib()
    L.mds_set_wait_limit_ns.argtypes = [ctypes.c_ulonglong]
    L.mds_set_wait_limit_ns.restype = None
    L.mds_set_wait_limit_ns(int(ns))


def mds_inject_alloc_failures(count: int):
    """Failure injection: the next ``count`` device allocations of model, plan
    or server creation fail (MDS_ERR_NOMEM)."""
    L = _lib()
    L.mds_inject_alloc_failures.argtypes = [_I]
    L.mds_inject_alloc_failures.restype = None
    L.mds_inject_alloc_failures(int(count))


def mds_set_tune_cache(path):
    """Tuning cache file (None turns it off): plans created with ``tune`` store
    the cluster size they measured there and later processes reuse it for the
    same batch shape on the same kind of GPU; process-wide."""
    L = _lib()
    L.mds_set_tune_cache.argtypes = [ctypes.c_char_p]
    L.mds_set_tune_cache.restype = _I
    _check(L.mds_set_tune_cache(None if path is None else os.fsencode(path)), "mds_set_tune_cache")


def mds_tune_cache_lookup(key: str) -> int:
    """The value stored under ``key`` (0 when absent or the cache is off)."""
    L = _lib()
    L.mds_tune_cache_lookup.argtypes = [ctypes.c_char_p, _P]
    L.mds_tune_cache_lookup.restype = _I
    v = ctypes.c_int(0)
    _check(L.mds_tune_cache_lookup(key.encode(), ctypes.byref(v)), "mds_tune_cache_lookup")
    return v.value


def mds_tune_cache_store(key: str, value: int):
    """Adds or replaces the entry ``key`` of the tuning cache."""
    L = _lib()
    L.mds_tune_cache_store.argtypes = [ctypes.c_char_p, _I]
    L.mds_tune_cache_store.restype = _I
    _check(L.mds_tune_cache_store(key.encode(), int(value)), "mds_tune_cache_store")


def mds_embed_new_static(model: Model, Ynew, stream=None):
    """mds_embed_new without any device allocation: scratch comes from a fixed
    array inside the library, so the only tensors created here are the
    outputs (pass ``out`` to avoid even that).  For callers that must not
    allocate device memory while embedding; see include/gbmds.h."""
    dt = _data(Ynew)
    m = Ynew.shape[0]
    info = model.info()
    L = _lib()
    L.mds_embed_new_static.argtypes = [_P, _P, _I, _I64, _P, _P]
    L.mds_embed_new_static.restype = _I
    st = stream if stream is not None else torch.cuda.current_stream(Ynew.device)
    o = MdsOpts(prec=PREC[info["prec"]], stream=ctypes.c_void_p(st.cuda_stream), workspace=None,
                workspace_bytes=0)
    X = torch.empty((m, info["r"]), dtype=_xdtype(info["prec"]), device=Ynew.device)
    _check(L.mds_embed_new_static(model.handle, _ptr(Ynew), dt, m, ctypes.byref(o), _ptr(X)),
           "mds_embed_new_static")
    return X


def mds_embed_new_static_capacity() -> int:
    L = _lib()
    L.mds_embed_new_static_capacity.restype = _SZ
    return L.mds_embed_new_static_capacity()


class MdsServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("flags", ctypes.c_int32), ("slot_bytes", ctypes.c_size_t),
                ("max_batch_rows", ctypes.c_int64)]


class MdsServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("rows", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("max_in_flight", ctypes.c_int32), ("slots", ctypes.c_int32)]


def _server_lib():
    L = _lib()
    if not getattr(L, "_server_sigs", False):
        for name, res, args in [
            ("mds_server_create", _I, [_P, _I, _P, _P]),
            ("mds_server_submit", _I, [_P, _I, _P, _I, _I64, _P, _P]),
            ("mds_server_wait", _I, [_P, ctypes.c_uint64, _D, _P, _P]),
            ("mds_server_get_stats", _I, [_P, _P]),
            ("mds_server_destroy", _I, [_P]),
        ]:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        L._server_sigs = True
    return L


class Server:
    """Continuous-batching embed server over resident models (mds_server_*).

    ``submit`` takes a CPU tensor of rows (pinned memory lets copies overlap)
    and returns a ticket; ``wait`` returns the CPU result tensor and the
    request's latency in ms.  Tensors are kept alive until their request is
    waited for."""

    def __init__(self, models, slots=4, slot_bytes=64 << 20, max_batch_rows=0):
        L = _server_lib()
        self.models = list(models)
        self.info = [m.info() for m in self.models]
        arr = (ctypes.c_void_p * len(self.models))(*[m.handle.value for m in self.models])
        o = MdsServerOpts(slots=slots, flags=0, slot_bytes=slot_bytes, max_batch_rows=max_batch_rows)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.models[0].device):
            _check(L.mds_server_create(arr, len(self.models), ctypes.byref(o), ctypes.byref(h)),
                   "mds_server_create")
        self.handle = h
        self._live = {}

    def submit(self, model: int, Y, out=None) -> int:
        if not (isinstance(Y, torch.Tensor) and not Y.is_cuda and Y.dim() == 2 and Y.is_contiguous()):
            raise ValueError("rows must be a contiguous 2-D CPU tensor")
        if Y.dtype not in DTYPE:
            raise ValueError(f"unsupported dtype {Y.dtype}")
        if not 0 <= model < len(self.info):
            raise ValueError(f"model index {model} out of range 0..{len(self.info) - 1}")
        inf = self.info[model]
        if Y.shape[1] != inf["d"]:
            raise ValueError(f"model {model} has d={inf['d']}, rows have {Y.shape[1]}")
        if out is None:
            out = torch.empty((Y.shape[0], inf["r"]), dtype=_xdtype(inf["prec"]), pin_memory=Y.is_pinned())
        t = ctypes.c_uint64()
        _check(_server_lib().mds_server_submit(self.handle, model, _ptr(Y), DTYPE[Y.dtype], Y.shape[0], _ptr(out),
                                               ctypes.byref(t)), "mds_server_submit")
        self._live[t.value] = (Y, out)
        return t.value

    def wait(self, ticket: int, timeout: float = 120.0):
        st, lat = ctypes.c_int(), ctypes.c_double()
        _check(_server_lib().mds_server_wait(self.handle, ticket, timeout, ctypes.byref(st), ctypes.byref(lat)),
               "mds_server_wait")
        _, out = self._live.pop(ticket)
        _check(st.value, "mds_server request")
        return out, lat.value

    def stats(self) -> dict:
        s = MdsServerStats()
        _check(_server_lib().mds_server_get_stats(self.handle, ctypes.byref(s)), "mds_server_get_stats")
        return {k: getattr(s, k) for k, _ in MdsServerStats._fields_}

    def close(self):
        if self.handle and self.handle.value:
            _check(_server_lib().mds_server_destroy(self.handle), "mds_server_destroy")
            self.handle = ctypes.c_void_p(0)
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DcPlan:
    """Divide-and-conquer plan (mds_dc_plan_*): fixed shapes, own workspace,
    the whole launch sequence replayed as one CUDA graph; ``tune=True`` makes
    the first ``execute`` pick the eigen-solver cluster size by timing."""

    def __init__(self, n, d, dtype, part_ptr, c, r, prec="f32", tune=True, cluster=0, device="cuda",
                 full_matvec=False, eig_tol=0.0):
        L = _lib()
        for name, res, args in [
            ("mds_dc_plan_create", _I, [_I64, _I, _I, _I, _P, _I, _I, _P, _I, _P]),
            ("mds_dc_plan_execute", _I, [_P, _P, _P, _P, _P, _P, _P]),
            ("mds_dc_plan_execute_host", _I, [_P, _P, _P, _P, _P, _P, _P]),
            ("mds_dc_plan_info", _I, [_P, _P, _P, _P]),
            ("mds_dc_plan_destroy", None, [_P]),
        ]:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        self.device = torch.device(device)
        self.ptr = np.ascontiguousarray(np.asarray(part_ptr, dtype=np.int64))
        self.p = len(self.ptr) - 1
        self.n, self.d, self.r, self.prec = n, d, r, prec
        o = MdsOpts(prec=PREC[prec], cluster=cluster, flags=FLAG_FULL_MATVEC if full_matvec else 0,
                    eig_tol=eig_tol)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.mds_dc_plan_create(n, d, DTYPE[dtype], self.p, self.ptr.ctypes.data_as(ctypes.c_void_p), c, r,
                                        ctypes.byref(o), 1 if tune else 0, ctypes.byref(h)), "mds_dc_plan_create")
        self.handle = h

    def execute(self, Y, anchors, part_own, X=None, var=None, stream=None):
        _data(Y)
        if X is None:
            X = torch.zeros((self.n, self.r), dtype=_xdtype(self.prec), device=Y.device)
        if var is None:
            var = torch.empty(self.r, dtype=torch.float64, device=Y.device)
        st = stream if stream is not None else torch.cuda.current_stream(Y.device)
        _check(_lib().mds_dc_plan_execute(self.handle, _ptr(Y), _ptr(part_own), _ptr(anchors), _ptr(X), _ptr(var),
                                          ctypes.c_void_p(st.cuda_stream)), "mds_dc_plan_execute")
        return X, var

    def execute_host(self, Y, anchors, part_own, X=None, var=None, stream=None):
        """The same run on host data: ``Y``, ``anchors`` and ``part_own`` are
        CPU tensors (pin them for asynchronous copies); returns CPU tensors
        (X pinned unless given).  The plan copies into device buffers it
        owns, replays its graph, and copies the results back."""
        if not (isinstance(Y, torch.Tensor) and not Y.is_cuda and Y.dim() == 2 and Y.is_contiguous()):
            raise ValueError("data must be a contiguous 2-D CPU tensor")
        anc = torch.as_tensor(anchors, dtype=torch.int64).contiguous()
        own = torch.as_tensor(part_own, dtype=torch.int64).contiguous()
        if anc.is_cuda or own.is_cuda:
            raise ValueError("anchors and part_own must be CPU tensors")
        if X is None:
            X = torch.empty((self.n, self.r), dtype=_xdtype(self.prec), pin_memory=True)
        if var is None:
            var = torch.empty(self.r, dtype=torch.float64)
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check(_lib().mds_dc_plan_execute_host(self.handle, _ptr(Y), _ptr(own), _ptr(anc), _ptr(X), _ptr(var),
                                               ctypes.c_void_p(st.cuda_stream)), "mds_dc_plan_execute_host")
        return X, var

    def info(self):
        cs, nodes = ctypes.c_int(), ctypes.c_int64()
        trials = (ctypes.c_double * 17)()
        _check(_lib().mds_dc_plan_info(self.handle, ctypes.byref(cs), ctypes.byref(nodes), trials), "mds_dc_plan_info")
        return {"cluster": cs.value, "graph_nodes": nodes.value,
                "trial_ms": {i: trials[i] for i in range(17) if trials[i] > 0}}

    def close(self):
        if self.handle and self.handle.value:
            _lib().mds_dc_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
