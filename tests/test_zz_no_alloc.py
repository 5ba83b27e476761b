"""The allocation-free embedding entry point (mds_embed_new_static).

Some callers must not allocate device memory while they embed new points
(their device memory is reserved by another allocator, or allocation is
forbidden inside their serving loop).  mds_embed_new_static serves them from
a fixed scratch array inside the library.  These tests check, through the C
ABI, that two calls in a row give the same result as mds_embed_new within
the FP32/FP64 tolerances used elsewhere, and that an oversized request is
refused before any work is done.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-5, "bf16": 2e-3}


@pytest.fixture(scope="module")
def gb():
    from paper_2007_11919_gb300 import build
    build.build()
    import paper_2007_11919_gb300 as G
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return G


@pytest.mark.parametrize("prec", ["f32", "f64", "bf16"])
def test_static_matches_allocating_entry_point(gb, prec):
    """BF16 models also stage the rounded rows in the array; FP32/FP64 models
    only the row norms."""
    from paper_2007_11919_gb300 import mds as M
    dt = np.float64 if prec == "f64" else np.float32
    Y = W.gaussian_dominant(4000, 40, 5, seed=31, dtype=dt)
    idx = W.landmarks(4000, 300, seed=31)
    _, _, model = gb.mds_interpolate(torch.from_numpy(Y).cuda(), torch.from_numpy(idx).cuda(), 5, prec,
                                     want_model=True)
    batches = [W.gaussian_dominant(1500, 40, 5, seed=32, dtype=dt), W.gaussian_dominant(777, 40, 5, seed=33, dtype=dt)]
    for Yn in batches:                                   # two calls in a row
        Yd = torch.from_numpy(Yn).cuda()
        ref = gb.mds_embed_new(model, Yd).double().cpu().numpy()
        got = M.mds_embed_new_static(model, Yd).double().cpu().numpy()
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= TOL[prec] * scale


def test_static_rejects_oversized_request(gb):
    from paper_2007_11919_gb300 import mds as M
    Y = W.gaussian_dominant(2000, 16, 3, seed=34, dtype=np.float32)
    idx = W.landmarks(2000, 200, seed=34)
    _, _, model = gb.mds_interpolate(torch.from_numpy(Y).cuda(), torch.from_numpy(idx).cuda(), 3, "f32",
                                     want_model=True)
    cap = M.mds_embed_new_static_capacity()
    rows = cap // 8 + 1024                                # norms alone exceed the array
    big = torch.zeros((rows, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(gb.MdsError) as e:
        M.mds_embed_new_static(model, big)
    assert e.value.status == 8
