"""The one-warp-per-pair forward (small bodies): the same manifold as the one-CTA-per-pair
kernel, its records drive the adjoint, and both agree with the oracle."""
import numpy as np
import pytest
import torch

import synth
from _parity import check_forward, check_grad

pytestmark = pytest.mark.gpu


def _engine_with(w, extra=None):
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    eng = Engine(0)
    ids = eng.add_geometries(w.geoms)
    if extra is not None:           # a large geometry moves the context off the warp path
        eng.add_geometries([extra])
    return eng, workload_tensors(w, id_map=ids)


def test_warp_path_equals_cta_path():
    """Box-box pairs in a context of boxes only (the warp path by default) and in one that
    also holds a 64-point hull (the CTA path): the same manifold, and the oracle's."""
    from paper_2602_20304_gb300 import api
    w = synth.make_config(1, 512)
    big = synth.hull_from_points(np.random.default_rng(0).normal(size=(64, 3)))
    e1, (pg, poses, dims, tau) = _engine_with(w)
    e2, t2 = _engine_with(w, big)
    try:
        assert api.cm_get_launch_shape(e1.ctx, w.n_pairs)[0] > 0
        o1 = e1.forward(pg, poses, dims, tau).cpu().numpy()
        o2 = e2.forward(*t2).cpu().numpy()
        e1.check()
        e2.check()
        print("warp vs CTA path, largest difference", float(np.abs(o1 - o2).max()))
        assert np.abs(o1 - o2).max() <= 2e-6
        idx = np.arange(0, w.n_pairs, 8)
        check_forward(o1[idx].astype(np.float64), w, e1.params(), idx, what="warp path")
    finally:
        e1.close()
        e2.close()


def test_warp_path_records_drive_the_adjoint():
    """A forward+backward plan of 256 box-box pairs (warp forward writing the records,
    record-driven adjoint) against the oracle's gradients, and the same gradients as the
    adjoint that recomputes the forward."""
    from paper_2602_20304_gb300 import api
    w = synth.make_config(1, 256)
    eng, (pg, poses, dims, tau) = _engine_with(w)
    try:
        params = eng.params()
        out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
        go = torch.randn(out.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
        gp, gd = torch.empty_like(poses), torch.empty_like(dims)
        plan = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
        try:
            api.cm_plan_launch(plan)
            torch.cuda.synchronize()
        finally:
            api.cm_plan_destroy(plan)
        eng.check()
        rgp, rgd = eng.backward(pg, poses, dims, tau, go, params)
        a = torch.cat([gp, gd], 1).double()
        b = torch.cat([rgp, rgd], 1).double()
        rel = ((a - b).abs().amax(1) / b.abs().amax(1).clamp_min(1e-12)).max().item()
        print("records vs recompute on the warp path, worst per-pair relative", rel)
        assert rel <= 1e-3
        gi = np.arange(0, w.n_pairs, 16)
        got = np.concatenate([gp.cpu().numpy(), gd.cpu().numpy()], 1)[gi].astype(np.float64)
        check_grad(got, w, params, go.cpu().numpy()[gi].astype(np.float64), gi, what="warp-path plan gradients")
        check_forward(out.cpu().numpy()[gi].astype(np.float64), w, params, gi, what="warp-path plan forward")
    finally:
        eng.close()


def test_warp_path_autotuned_and_empty_flags():
    """The autotuner's warp shapes and the vertex-only mode on the warp path."""
    from paper_2602_20304_gb300 import api
    w = synth.make_config(1, 300)
    eng, (pg, poses, dims, tau) = _engine_with(w)
    try:
        params = eng.params()
        out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
        api.cm_autotune(eng.ctx, pg, poses, dims, tau, params, out)
        o = eng.forward(pg, poses, dims, tau, params).cpu().numpy()
        idx = np.arange(0, w.n_pairs, 10)
        check_forward(o[idx].astype(np.float64), w, params, idx, what="autotuned warp path")
        p1 = eng.params(flags=1, K=4)
        o1 = eng.forward(pg, poses, dims, tau, p1).cpu().numpy()
        check_forward(o1[idx].astype(np.float64), w, p1, idx, what="warp path, vertex contacts only")
        eng.check()
    finally:
        eng.close()
