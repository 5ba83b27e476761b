"""Serving loop (mds_server_*): continuous batching of embed requests onto
resident models, checked against the oracle's Eq. (2) and against each
request run alone."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL_BF16 = 2e-3


@pytest.fixture(scope="module")
def gb():
    from paper_2007_11919_gb300 import build
    build.build()
    import paper_2007_11919_gb300 as G
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return G


@pytest.fixture(scope="module")
def resident(gb):
    """The three resident BF16 models of the serving workload, plus the
    oracle's model of the same landmarks."""
    from paper_2007_11919_gb300 import mds as M
    w = W.SERVE_BF16
    Y0 = W.make_data(w, seed=21, n=6000)
    models, oracle_models = [], []
    for k, (l, r) in enumerate(W.SERVE_MODELS):
        idx = W.landmarks(len(Y0), l, seed=100 + k)
        _, _, m = M.mds_interpolate(torch.from_numpy(Y0).cuda(), torch.from_numpy(idx).cuda(), r, "bf16",
                                    want_model=True)
        models.append(m)
        _, _, ex = O.interpolation_mds(Y0[idx], np.arange(l), r)
        ex["L"] = Y0[idx].astype(np.float64)
        oracle_models.append(ex)
    return models, oracle_models


def _requests(count, hi, seed):
    rng = np.random.default_rng(seed)
    _, sizes = W.serve_requests(count, 1, hi, rate_per_s=1.0, seed=seed)
    which = rng.integers(0, len(W.SERVE_MODELS), size=count)
    Ynew = W.make_data(W.SERVE_BF16, seed=seed + 7, n=int(sizes.sum()))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rows = [torch.from_numpy(Ynew[offs[i]:offs[i + 1]]).pin_memory() for i in range(count)]
    return which, rows


def test_alone_equals_mix_and_oracle(gb, resident):
    from paper_2007_11919_gb300.mds import Server
    models, oracle_models = resident
    which, rows = _requests(48, 6000, seed=3)
    with Server(models, slots=4) as srv:
        alone = []
        for k, Y in zip(which, rows):
            X, _ = srv.wait(srv.submit(int(k), Y))
            alone.append(X.clone())
        before = srv.stats()
        tickets = [srv.submit(int(k), Y) for k, Y in zip(which, rows)]   # one burst
        mix = [srv.wait(t) for t in tickets]
        after = srv.stats()
    for a, (b, lat) in zip(alone, mix):
        assert torch.equal(a, b)            # same bits alone and in the mix
        assert lat > 0
    assert after["requests"] - before["requests"] == len(rows)
    assert after["batches"] - before["batches"] < len(rows)    # requests shared launches
    assert after["max_in_flight"] >= 2                          # batches overlapped
    for k, om in enumerate(oracle_models):
        sel = [i for i in range(len(rows)) if which[i] == k]
        if not sel:
            continue
        got = torch.cat([alone[i] for i in sel]).double().numpy()
        ref = O.embed_new(om, torch.cat([rows[i] for i in sel]).double().numpy())
        assert O.aligned_rel_error(got, ref) < TOL_BF16


def test_split_requests_match(gb, resident):
    """A slot arena smaller than a request splits it across batches; the rows
    are the same as in one launch."""
    from paper_2007_11919_gb300.mds import Server
    models, _ = resident
    which, rows = _requests(12, 20_000, seed=5)
    with Server(models, slots=2) as big:
        ref = [big.wait(big.submit(int(k), Y))[0].clone() for k, Y in zip(which, rows)]
    with Server(models, slots=3, slot_bytes=1 << 20) as small:
        tickets = [small.submit(int(k), Y) for k, Y in zip(which, rows)]
        got = [small.wait(t)[0] for t in tickets]
        st = small.stats()
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    big_rows = max(Y.shape[0] for Y in rows)
    assert big_rows > 2000 and st["batches"] > len(rows)   # 1 MiB holds fewer rows than the largest request


def test_pageable_and_errors(gb, resident):
    from paper_2007_11919_gb300.mds import MdsError, Server
    models, _ = resident
    Y = torch.from_numpy(W.make_data(W.SERVE_BF16, seed=9, n=300))      # pageable
    with Server(models[:1], slots=1) as srv:
        X, _ = srv.wait(srv.submit(0, Y))
        assert X.shape == (300, W.SERVE_MODELS[0][1]) and torch.isfinite(X).all()
        with pytest.raises(ValueError):
            srv.submit(0, Y[:, :50].contiguous())
        with pytest.raises(ValueError):
            srv.submit(3, Y)
        import ctypes
        from paper_2007_11919_gb300.mds import _ptr, _server_lib
        t = ctypes.c_uint64()
        out = torch.empty(300, 2)
        assert _server_lib().mds_server_submit(srv.handle, 3, _ptr(Y), 1, 300, _ptr(out), ctypes.byref(t)) == 1
        with pytest.raises(MdsError):
            srv.wait(123456)
