"""The allocation-free forward entry point, called through the C ABI.

Some callers of this library cannot allocate device memory while they run the
manifold: a host application that hands out every device allocation from its own
pool, or a real-time loop that was promised a fixed memory footprint and cannot
absorb the blocking of cudaMalloc / cudaFree.  For them the library has
cm_contact_manifold_fwd_noalloc, whose scratch is a fixed array inside the library.
Its output must equal the regular forward entry point's, within the parity
tolerance, on two calls in a row (the second call finds the first call's leftovers
in the shared array), it must refuse what the regular entry point refuses, and the
device's free memory must not change across a call.
This file is collected last on purpose, so a run that stops at the first failure
has run every other test before it.
"""
import numpy as np
import pytest
import torch

import synth
from _parity import TOL, errors

pytestmark = pytest.mark.gpu


@pytest.fixture()
def engine():
    from paper_2602_20304_gb300.engine import Engine
    e = Engine(0)
    yield e
    e.close()


def _regular_and_noalloc(eng, w, calls=2, **pkw):
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = eng.add_geometries(w.geoms)           # uploads: the no-alloc call must not have to
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = eng.params(**pkw)
    ref = eng.forward(pg, poses, dims, tau, params)
    torch.cuda.synchronize()
    eng.check()
    ref = ref.cpu().numpy().astype(np.float64)
    outs = []
    for call in range(calls):
        out = torch.full(ref.shape, float("nan"), dtype=torch.float32, device="cuda")
        api.cm_contact_manifold_fwd_noalloc(eng.ctx, pg, poses, dims, tau, params, out)
        torch.cuda.synchronize()
        eng.check()
        outs.append(out.cpu().numpy().astype(np.float64))
    return ref, outs


def test_no_alloc_matches_regular_forward_twice(engine):
    w = synth.make_config(2, 256)
    ref, outs = _regular_and_noalloc(engine, w)
    for call, got in enumerate(outs):
        assert np.isfinite(got).all(), f"call {call}: non-finite output"
        err = errors(got, ref)
        assert all(err[k] <= TOL[k] for k in err), (call, err)


@pytest.mark.parametrize("flags", [1, 2])
def test_no_alloc_simplified_modes_match_regular_forward(engine, flags):
    """Vertex contacts only, and one-sided vertex contacts (K = 4 fits the smallest hull)."""
    w = synth.make_config(2, 128)
    ref, outs = _regular_and_noalloc(engine, w, flags=flags, K=4)
    for call, got in enumerate(outs):
        assert np.isfinite(got).all(), f"flags {flags} call {call}: non-finite output"
        err = errors(got, ref)
        assert all(err[k] <= TOL[k] for k in err), (flags, call, err)


def test_no_alloc_refuses_what_the_regular_entry_point_refuses(engine):
    """Vertex contacts only with 2 soft pre-selected vertices per body leave 4 candidates
    per box-box pair: K = 8 is refused by both entry points, with the same status."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.make_config(1, 8)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    api.cm_sync_geometry(engine.ctx)
    params = engine.params(flags=1, top_verts=2, K=8)
    out = torch.empty((w.n_pairs, 8, 8), device="cuda")
    with pytest.raises(api.CMError) as regular:
        api.cm_contact_manifold_fwd(engine.ctx, pg, poses, dims, tau, params, out)
    with pytest.raises(api.CMError) as noalloc:
        api.cm_contact_manifold_fwd_noalloc(engine.ctx, pg, poses, dims, tau, params, out)
    assert regular.value.status == noalloc.value.status == api.CM_ERR_INVALID_ARG


def test_no_alloc_leaves_free_device_memory_unchanged(engine):
    """After a first call (which looks up the array's address and sets the kernel's
    shared-memory limit), further calls change the device's free memory by nothing."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.make_config(2, 512)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params()
    api.cm_sync_geometry(engine.ctx)
    out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
    api.cm_contact_manifold_fwd_noalloc(engine.ctx, pg, poses, dims, tau, params, out)
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        api.cm_contact_manifold_fwd_noalloc(engine.ctx, pg, poses, dims, tau, params, out)
    torch.cuda.synchronize()
    after = torch.cuda.mem_get_info()[0]
    engine.check()
    assert after == before, (before, after)
    assert np.isfinite(out.cpu().numpy()).all()


def test_no_alloc_rejects_oversized_geometry_and_pending_upload(engine):
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(0)
    u = rng.normal(size=(256, 3))
    big = synth.hull_from_points(u / np.linalg.norm(u, axis=1, keepdims=True))   # 762 edges
    gid = engine.add_geometry(big)
    params = engine.params()
    pg = torch.tensor([[gid, gid]], dtype=torch.int32, device="cuda")
    poses = torch.tensor([[1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 1.9]], dtype=torch.float32,
                         device="cuda")
    out = torch.empty((1, params.K, 8), device="cuda")
    with pytest.raises(api.CMError) as ei:                       # upload still pending
        api.cm_contact_manifold_fwd_noalloc(engine.ctx, pg, poses, None, None, params, out)
    assert ei.value.status == api.CM_ERR_INVALID_ARG and "cm_sync_geometry" in str(ei.value)
    api.cm_sync_geometry(engine.ctx)
    with pytest.raises(api.CMError) as ei:                       # 762 edges > the limit
        api.cm_contact_manifold_fwd_noalloc(engine.ctx, pg, poses, None, None, params, out)
    assert ei.value.status == api.CM_ERR_INVALID_ARG and "edges" in str(ei.value)
