"""Batching layer: size-ordered persistent launches, autotuned launch shapes and
CUDA-graph plans give the same manifold as one launch per pair."""
import numpy as np
import pytest
import torch

import synth
from _parity import check_forward, check_grad, contact_share

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    eng = Engine(0)
    w = synth.config_mixed(n=96, seed=123)
    w.tau[:] = 1e-2
    ids = eng.add_geometries(w.geoms)
    yield eng, w, workload_tensors(w, id_map=ids)
    eng.close()


def test_uneven_batch_equals_per_pair_launches(setup):
    eng, w, (pg, poses, dims, tau) = setup
    batched = eng.forward(pg, poses, dims, tau).cpu().numpy()
    single = np.stack([eng.forward(pg[i:i + 1], poses[i:i + 1], dims[i:i + 1], tau[i:i + 1]).cpu().numpy()[0]
                       for i in range(w.n_pairs)])
    eng.check()
    assert np.abs(batched - single).max() <= 1e-6


def test_autotune_then_plan_replay(setup):
    from paper_2602_20304_gb300 import api
    eng, w, (pg, poses, dims, tau) = setup
    params = eng.params()
    ref = eng.forward(pg, poses, dims, tau, params).clone()
    out = torch.empty_like(ref)
    go = torch.randn_like(ref)
    gp = torch.empty_like(poses)
    gd = torch.empty_like(dims)
    api.cm_autotune(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
    shape_f = api.cm_get_launch_shape(eng.ctx, w.n_pairs, False)
    shape_b = api.cm_get_launch_shape(eng.ctx, w.n_pairs, True)
    assert shape_f[0] in (128, 256, 512) and shape_b[0] in (128, 256)
    # the plan's adjoint reads the forward's records, as the autograd path does
    saved = eng.forward_save(pg, poses, dims, tau, params)[1]
    ref_gp, ref_gd = eng.backward(pg, poses, dims, tau, go, params, saved=saved)
    # a plan captures ordering + forward + adjoint; replay it twice with new poses in between
    poses_buf = poses.clone()
    plan = api.cm_plan_create(eng.ctx, pg, poses_buf, dims, tau, params, out, go, gp, gd)
    try:
        api.cm_plan_launch(plan)
        torch.cuda.synchronize()
        assert torch.allclose(out, ref, atol=1e-6, rtol=0)
        # the adjoint sums with atomics: two launches agree to the rounding of those sums,
        # held per pair relative to the pair's largest gradient component
        a = torch.cat([gp, gd], 1).double()
        b = torch.cat([ref_gp, ref_gd], 1).double()
        rel = ((a - b).abs().amax(1) / b.abs().amax(1).clamp_min(1e-12)).max().item()
        print("plan vs direct adjoint, worst per-pair relative difference", rel)
        assert rel <= 1e-4
        moved = poses.clone()
        moved[:, 4:7] += 0.01
        moved[:, 11:14] += 0.01                     # rigid shift of both bodies
        poses_buf.copy_(moved)
        api.cm_plan_launch(plan)
        torch.cuda.synchronize()
        eager = eng.forward(pg, moved, dims, tau, params)
        assert torch.allclose(out, eager, atol=1e-6, rtol=0)
        eng.add_geometry(w.geoms[0])                # new geometry invalidates the plan
        api.cm_sync_geometry(eng.ctx)
        with pytest.raises(api.CMError):
            api.cm_plan_launch(plan)
    finally:
        api.cm_plan_destroy(plan)
    eng.check()


def test_plan_matches_oracle_on_mixed_batch(setup):
    from paper_2602_20304_gb300 import api
    eng, w, (pg, poses, dims, tau) = setup
    params = eng.params()
    out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
    plan = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out)
    try:
        api.cm_plan_launch(plan)
        torch.cuda.synchronize()
    finally:
        api.cm_plan_destroy(plan)
    idx = np.arange(0, w.n_pairs, 6)
    check_forward(out.cpu().numpy()[idx], w, params, idx, what="plan")


def test_full_size_uneven_batch_sampled():
    """65536 uneven pairs (hull pool of 4096, mixed primitives, tau in {1e-3, 1e-2, 1e-1}) in one
    graph-replayed step with the adjoint; 120 seeded pairs against the oracle's values and 24
    (eight per tau) against its gradients, every one under the per-pair bar."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    w = synth.config_mixed_pooled()
    eng = Engine(0)
    try:
        ids = eng.add_geometries(w.geoms)
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        params = eng.params()
        out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
        go = torch.randn_like(out)
        gp, gd = torch.empty_like(poses), torch.empty_like(dims)
        plan = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
        try:
            api.cm_plan_launch(plan)
            torch.cuda.synchronize()
        finally:
            api.cm_plan_destroy(plan)
        eng.check()
        o, gpn, gdn, gon = out.cpu().numpy(), gp.cpu().numpy(), gd.cpu().numpy(), go.cpu().numpy()
        assert np.isfinite(o).all() and np.isfinite(gpn).all() and np.isfinite(gdn).all()
        rng = np.random.default_rng(4)
        idx = rng.choice(w.n_pairs, 120, replace=False)
        check_forward(o[idx], w, params, idx, what="65536 uneven sample")
        for tv in (1e-3, 1e-2):
            sel = idx[np.isclose(w.tau[idx], tv)]
            share = contact_share(w, sel, frac_tau=0.5)
            print(f"tau={tv}: pairs with a score above tau / 2", share, "of", len(sel))
            assert share >= 0.6
        gi = np.concatenate([idx[np.isclose(w.tau[idx], tv)][:8] for tv in (1e-3, 1e-2, 1e-1)])
        assert len(gi) == 24
        got = np.concatenate([gpn[gi], gdn[gi]], 1)
        print(check_grad(got, w, params, gon[gi], gi, what="65536 uneven gradient sample"))
    finally:
        eng.close()


@pytest.mark.parametrize("cfg", [2, 3])
def test_full_size_autotuned_step_sampled(cfg):
    """The benchmark's launch configuration at full size: 4096 hull-vs-primitive pairs or
    1024 box-vs-hull32 pairs, autotuned launch shapes, one graph-replayed forward+adjoint
    step; 100 seeded pairs against the oracle's values and 16 against its gradients."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    w = synth.make_config(cfg)
    eng = Engine(0)
    try:
        ids = eng.add_geometries(w.geoms)
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        params = eng.params()
        out = torch.empty((w.n_pairs, params.K, 8), device="cuda")
        go = torch.randn(out.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(cfg))
        gp, gd = torch.empty_like(poses), torch.empty_like(dims)
        api.cm_autotune(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
        plan = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, params, out, go, gp, gd)
        try:
            for _ in range(2):
                api.cm_plan_launch(plan)
            torch.cuda.synchronize()
        finally:
            api.cm_plan_destroy(plan)
        eng.check()
        o, gpn, gdn, gon = out.cpu().numpy(), gp.cpu().numpy(), gd.cpu().numpy(), go.cpu().numpy()
        assert np.isfinite(o).all() and np.isfinite(gpn).all() and np.isfinite(gdn).all()
        idx = np.random.default_rng(10 + cfg).choice(w.n_pairs, 100, replace=False)
        check_forward(o[idx], w, params, idx, what=f"config {cfg} sample")
        gi = idx[:16]
        check_grad(np.concatenate([gpn[gi], gdn[gi]], 1), w, params, gon[gi], gi, what=f"config {cfg} gradients")
    finally:
        eng.close()
