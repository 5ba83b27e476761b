"""Error paths of the library on the GPU, made to run without faulting, trapping
or hanging anything: an eigen-solver step cap (MDS_ERR_NOCONV), a team
grid-barrier wait whose limit the host shortens so that it gives up
(MDS_ERR_TIMEOUT, after which the context stays usable and the same call
succeeds), and device allocations that the host makes fail (MDS_ERR_NOMEM).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    from paper_2007_11919_gb300 import build
    build.build()
    import paper_2007_11919_gb300 as G
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return G


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_step_cap_is_noconv(gb):
    """Eight Lanczos steps cannot resolve ten close eigenvalues: the status word
    of the problem says so, for a single problem and for a batch of parts."""
    Y = W.gaussian_dominant(2000, 40, 10, seed=1)
    with pytest.raises(gb.MdsError) as e:
        gb.mds_classical(dev(Y), 10, "f64", max_steps=12)
    assert e.value.status == 5
    part = W.partitions_uneven(6000, 20, 800, 1200, seed=2)
    Yd = W.gaussian_dominant(6000, 40, 10, seed=2, dtype=np.float32)
    with pytest.raises(gb.MdsError) as e:
        gb.mds_divide_conquer(dev(Yd), dev(part.anchors), part.ptr, dev(part.own), 10, "f32", max_steps=12)
    assert e.value.status == 5
    X, lam = gb.mds_classical(dev(Y), 10, "f64")                     # the default cap converges
    assert np.all(np.isfinite(X.cpu().numpy()))


def test_team_barrier_timeout_then_recovery(gb):
    """A 1 ns limit on the team's grid-barrier waits: a cluster that arrives
    before the others gives up at once, the team leaves the solve together and
    the call returns MDS_ERR_TIMEOUT.  With the default limit restored the same
    calls run to the oracle's answer on the same context."""
    from paper_2007_11919_gb300 import mds as M
    Y = W.gaussian_dominant(3000, 20, 4, seed=3)
    idx = W.landmarks(3000, 1500, seed=3)
    try:
        M.mds_set_wait_limit_ns(1)
        with pytest.raises(gb.MdsError) as e:
            gb.mds_classical(dev(Y), 4, "f64")
        assert e.value.status == 6
        with pytest.raises(gb.MdsError) as e:
            gb.mds_interpolate(dev(Y), dev(idx), 4, "f64")
        assert e.value.status == 6
    finally:
        M.mds_set_wait_limit_ns(0)
    X, lam = gb.mds_classical(dev(Y), 4, "f64")
    Xo, lo, _, _ = O.classical_mds(O.sq_dist(Y, Y), 4)
    assert O.aligned_rel_error(X.cpu().numpy(), Xo) < 1e-10
    Xi, _, _ = gb.mds_interpolate(dev(Y), dev(idx), 4, "f64")
    Xio, _, _ = O.interpolation_mds(Y, idx, 4)
    assert O.aligned_rel_error(Xi.cpu().numpy(), Xio) < 1e-10


def test_injected_allocation_failures(gb, tmp_path):
    """Model, plan and server creation return MDS_ERR_NOMEM when a device
    allocation fails (injected on the host), free what they had, and work once
    the injected failures are used up."""
    from paper_2007_11919_gb300 import mds as M
    Y = W.gaussian_dominant(3000, 16, 4, seed=4, dtype=np.float32)
    idx = W.landmarks(3000, 300, seed=4)
    try:
        for k in (1, 4):                       # the first and a later allocation of the model
            M.mds_inject_alloc_failures(k)
            with pytest.raises(gb.MdsError) as e:
                gb.mds_interpolate(dev(Y), dev(idx), 4, "f32", want_model=True)
            assert e.value.status == 2
            M.mds_inject_alloc_failures(0)
        _, _, model = gb.mds_interpolate(dev(Y), dev(idx), 4, "f32", want_model=True)
        path = str(tmp_path / "m.gbmds")
        model.save(path)
        M.mds_inject_alloc_failures(1)
        with pytest.raises(gb.MdsError) as e:
            gb.Model.load(path)
        assert e.value.status == 2
        part = W.partitions_uneven(3000, 10, 300, 400, seed=4)
        M.mds_inject_alloc_failures(1)
        with pytest.raises(gb.MdsError) as e:
            M.DcPlan(3000, 16, torch.float32, part.ptr, 10, 4, "f32", tune=False, cluster=2)
        assert e.value.status == 2
        M.mds_inject_alloc_failures(1)
        with pytest.raises(gb.MdsError) as e:
            M.Server([model], slots=2, slot_bytes=8 << 20)
        assert e.value.status == 2
    finally:
        M.mds_inject_alloc_failures(0)
    m2 = gb.Model.load(path)
    assert torch.equal(gb.mds_embed_new(m2, dev(Y[:64])), gb.mds_embed_new(model, dev(Y[:64])))
    plan = M.DcPlan(3000, 16, torch.float32, part.ptr, 10, 4, "f32", tune=False, cluster=2)
    X, _ = plan.execute(dev(Y), dev(part.anchors), dev(part.own))
    assert np.all(np.isfinite(X.cpu().numpy()))
    plan.close()
    with M.Server([model], slots=2, slot_bytes=8 << 20) as srv:
        out, _ = srv.wait(srv.submit(0, torch.from_numpy(Y[:100].copy())))
    assert torch.equal(out, gb.mds_embed_new(model, dev(Y[:100])).cpu())
