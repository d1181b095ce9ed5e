"""The allocation-free forward entry point, called through the C ABI.

It serves callers that may not allocate device memory while they run (inside a
CUDA stream capture, in a fixed-footprint real-time loop, or under a host that
owns all device memory): its scratch is a fixed array inside the library.  Its
output must equal the regular forward entry point's, on two calls in a row
(the second call finds the first call's leftovers in the shared array).
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
from _parity import TOL, errors

pytestmark = pytest.mark.gpu


def test_no_alloc_matches_regular_forward_twice():
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    eng = Engine(0)
    try:
        w = synth.make_config(2, 256)
        ids = eng.add_geometries(w.geoms)           # uploads: the no-alloc call must not have to
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        params = eng.params()
        ref = eng.forward(pg, poses, dims, tau, params)
        torch.cuda.synchronize()
        eng.check()
        ref = ref.cpu().numpy()
        for call in range(2):
            out = torch.full_like(torch.as_tensor(ref, device="cuda"), float("nan"))
            api.cm_contact_manifold_fwd_noalloc(eng.ctx, pg, poses, dims, tau, params, out)
            torch.cuda.synchronize()
            eng.check()
            got = out.cpu().numpy()
            assert np.isfinite(got).all(), f"call {call}: non-finite output"
            err = errors(got.astype(np.float64), ref.astype(np.float64))
            assert all(err[k] <= TOL[k] for k in err), (call, err)
    finally:
        eng.close()


def test_no_alloc_rejects_oversized_geometry_and_pending_upload():
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine
    eng = Engine(0)
    try:
        rng = np.random.default_rng(0)
        u = rng.normal(size=(256, 3))
        big = synth.hull_from_points(u / np.linalg.norm(u, axis=1, keepdims=True))   # 762 edges
        gid = eng.add_geometry(big)
        params = eng.params()
        pg = torch.tensor([[gid, gid]], dtype=torch.int32, device="cuda")
        poses = torch.tensor([[1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 1.9]], dtype=torch.float32,
                             device="cuda")
        out = torch.empty((1, params.K, 8), device="cuda")
        with pytest.raises(api.CMError) as ei:                       # upload still pending
            api.cm_contact_manifold_fwd_noalloc(eng.ctx, pg, poses, None, None, params, out)
        assert ei.value.status == api.CM_ERR_INVALID_ARG and "cm_sync_geometry" in str(ei.value)
        api.cm_sync_geometry(eng.ctx)
        with pytest.raises(api.CMError) as ei:                       # 762 edges > the limit
            api.cm_contact_manifold_fwd_noalloc(eng.ctx, pg, poses, None, None, params, out)
        assert ei.value.status == api.CM_ERR_INVALID_ARG and "edges" in str(ei.value)
    finally:
        eng.close()
