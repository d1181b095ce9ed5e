"""Forward parity of the CUDA library against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import synth
from _parity import check_forward, contact_share, errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    from paper_2602_20304_gb300.engine import Engine
    e = Engine(0)
    yield e
    e.close()


def run(engine, w, **pkw):
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params(**pkw)
    out = engine.forward(pg, poses, dims, tau, params)
    torch.cuda.synchronize()
    engine.check()
    return out.cpu().numpy().astype(np.float64), params


def test_box_box_all_pairs(engine):
    """1024 box-box poses, tau = 1e-2, K = 8: every pair against the oracle."""
    w = synth.make_config(1)
    gpu, params = run(engine, w)
    check_forward(gpu, w, params, what="box-box")
    share = contact_share(w, range(128), frac_tau=0.5)
    print("box-box: pairs with a score above tau / 2", share)
    assert share >= 0.6


def test_hull_vs_primitive_subset(engine):
    w = synth.make_config(2, 96)
    gpu, params = run(engine, w)
    check_forward(gpu, w, params, what="hull-vs-primitive")


def test_hull_vs_primitive_full_size_sampled(engine):
    """All 4096 pairs in one launch; 128 seeded pairs re-computed by the oracle, most of
    them in active contact."""
    w = synth.make_config(2)
    gpu, params = run(engine, w)
    idx = np.random.default_rng(0).choice(w.n_pairs, 128, replace=False)
    check_forward(gpu[idx], w, params, idx, what="hull-vs-primitive full-size sample")
    share = contact_share(w, idx, frac_tau=0.5)
    print("pairs with a score above tau / 2", share)
    assert share >= 0.6


def test_box_vs_sphere_hull_subset(engine):
    w = synth.make_config(3, 64)
    gpu, params = run(engine, w)
    check_forward(gpu, w, params, what="box-vs-hull32")


@pytest.mark.parametrize("tau", [1e-2, 1e-1])
def test_hull_vs_hull(engine, tau):
    """Both bodies hulls (each of 8..64 points), either one with more planes."""
    w = synth.config_hull_vs_hull(n=48, tau=tau)
    npl = np.array([g.n_planes for g in w.geoms])
    a, b = npl[w.pair_geoms[:, 0]], npl[w.pair_geoms[:, 1]]
    assert (a > b).any() and (b > a).any()
    gpu, params = run(engine, w)
    check_forward(gpu, w, params, what=f"hull-vs-hull tau={tau}")


@pytest.mark.parametrize("tau", [1e-3, 1e-2, 1e-1])
def test_mixed_sizes_per_tau(engine, tau):
    """Hulls of 8..256 points against all primitive kinds at each smoothing level; every
    pair within the fixed tolerance or its own one-ulp conditioning bound."""
    w = synth.config_mixed(n=48, seed=99)
    w.tau[:] = tau
    gpu, params = run(engine, w)
    check_forward(gpu, w, params, what=f"mixed tau={tau}")
    if tau <= 1e-2:
        assert contact_share(w, range(w.n_pairs), frac_tau=0.5) >= 0.6


@pytest.mark.parametrize("flags", [1, 2])
def test_simplification_flags(engine, flags):
    w = synth.make_config(2, 32)
    gpu, params = run(engine, w, flags=flags, K=4)
    check_forward(gpu, w, params, what=f"flags={flags}")


@pytest.mark.parametrize("K", [1, 3, 16])
def test_other_K(engine, K):
    w = synth.make_config(1, 64)
    gpu, params = run(engine, w, K=K)
    assert gpu.shape[1] == K
    check_forward(gpu, w, params, what=f"K={K}")


def test_swap_symmetry_on_gpu(engine):
    """Exchanging the bodies of every pair leaves the manifold unchanged."""
    w = synth.make_config(2, 64)
    a, params = run(engine, w)
    ws = w.subset(np.arange(w.n_pairs))
    ws.pair_geoms = w.pair_geoms[:, ::-1].copy()
    ws.poses = np.concatenate([w.poses[:, 7:], w.poses[:, :7]], axis=1).copy()
    ws.dims = np.concatenate([w.dims[:, 3:], w.dims[:, :3]], axis=1).copy()
    b, _ = run(engine, ws)
    # the oracle's manifold is swap-symmetric (pinned on the CPU), so the swapped batch is
    # held to the oracle of the original pairs under the same per-pair bar
    check_forward(b, w, params, what="swapped bodies")
    print("swapped vs original GPU", errors(a, b))


def test_invalid_geometry_id_sets_flag(engine):
    from paper_2602_20304_gb300 import api
    w = synth.make_config(1, 8)
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    pg[3, 1] = 10 ** 6
    out = engine.forward(pg, poses, dims, tau)
    with pytest.raises(api.CMError) as ei:
        engine.check()
    assert ei.value.status == api.CM_ERR_DEVICE and "pair 3" in str(ei.value)
    o = out.cpu().numpy()
    assert np.isnan(o[3]).all() and np.isfinite(np.delete(o, 3, axis=0)).all()
    engine.check()                                   # flag was cleared


def test_destroyed_geometry_acts_as_unknown_id():
    """After cm_destroy_geometry a pair naming the geometry gets NaN rows and the error
    flag while the other pairs are unchanged; a plan made before is refused."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    w = synth.make_config(1, 16)
    eng = Engine(0)
    try:
        ids = eng.add_geometries(w.geoms)
        spare = eng.add_geometries(w.geoms)[0]          # a second copy of the cube
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        pg[8:, 1] = int(spare)
        before = eng.forward(pg, poses, dims, tau).cpu().numpy()
        eng.check()
        plan = api.cm_plan_create(eng.ctx, pg, poses, dims, tau, eng.params(), torch.empty((16, 8, 8), device="cuda"))
        api.cm_destroy_geometry(eng.ctx, int(spare))
        with pytest.raises(api.CMError) as ei:
            api.cm_plan_launch(plan)
        assert ei.value.status == api.CM_ERR_INVALID_ARG
        api.cm_plan_destroy(plan)
        after = eng.forward(pg, poses, dims, tau).cpu().numpy()
        with pytest.raises(api.CMError) as ei:
            eng.check()
        assert ei.value.status == api.CM_ERR_DEVICE
        assert np.isnan(after[8:]).all()
        np.testing.assert_allclose(after[:8], before[:8], atol=1e-6, rtol=0)
        gp, _ = eng.backward(pg, poses, dims, tau, torch.ones((16, 8, 8), device="cuda"))
        g = gp.cpu().numpy()
        with pytest.raises(api.CMError):
            eng.check()
        assert np.isnan(g[8:]).all() and np.isfinite(g[:8]).all()
        eng.check()
    finally:
        eng.close()


def test_empty_and_argument_errors(engine):
    from paper_2602_20304_gb300 import api
    engine.add_geometries(synth.make_config(1, 2).geoms)
    z = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    out = engine.forward(z, torch.zeros((0, 14), device="cuda"))
    assert out.shape == (0, 8, 8)
    with pytest.raises(api.CMError):
        engine.forward(torch.zeros((1, 2), dtype=torch.int32, device="cuda"),
                       torch.zeros((1, 14), device="cuda"), params=engine.params(K=17))
    with pytest.raises(api.CMError):
        engine.forward(torch.zeros((1, 2), dtype=torch.int32, device="cuda"),
                       torch.zeros((1, 14), device="cuda"), params=engine.params(tau=0.0))


def test_library_built_hull_gives_the_same_manifold():
    """A hull registered from its points (the library builds mesh and planes) gives the
    manifold of the same hull registered from the input generator's mesh and planes, and
    both match the oracle."""
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    w = synth.make_config(2, 16)
    eng = Engine(0)
    try:
        ids = eng.add_geometries(w.geoms)
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        a = eng.forward(pg, poses, dims, tau).cpu().numpy()
        eng.check()
        # the same pairs with every hull rebuilt from its vertices by the library
        hull_ids = ids.copy()
        for j, g in enumerate(w.geoms):
            if g.kind == synth.KIND_HULL:
                hull_ids[j] = eng.add_hull(g.verts[:, :3].astype(np.float64))
        pg2, _, _, _ = workload_tensors(w, id_map=hull_ids)
        b = eng.forward(pg2, poses, dims, tau).cpu().numpy()
        eng.check()
        np.testing.assert_allclose(b, a, rtol=0, atol=2e-6)
        params = eng.params()
        check_forward(b.astype(np.float64), w, params, what="library-built hulls")
    finally:
        eng.close()


def test_library_cube_hull_equals_the_box_primitive():
    """The library's hull of the 8 corners of [-0.5, 0.5]^3 (6 facet planes, 12 edges) gives
    the BOX primitive's manifold against the same partners, and both meet the oracle."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    corners = 0.5 * np.array([[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)])
    w = synth.config_hull_vs_primitive(n=64, seed=31)
    box = synth.primitive_geometry(synth.KIND_BOX)
    eng = Engine(0)
    try:
        ids = eng.add_geometries([box] + w.geoms)
        hid = eng.add_hull(corners)
        info = api.cm_get_geometry(eng.ctx, hid)
        assert (len(info["verts"]), len(info["edges"]), len(info["planes"])) == (8, 12, 6)
        wb = w.subset(np.arange(w.n_pairs))
        wb.geoms = [box] + w.geoms
        wb.pair_geoms = np.stack([np.zeros(w.n_pairs, np.int32), 1 + w.pair_geoms[:, 1]], 1)
        wb.dims[:, :3] = 0.5
        pg, poses, dims, tau = workload_tensors(wb, id_map=ids)
        a = eng.forward(pg, poses, dims, tau).cpu().numpy().astype(np.float64)
        pg_h = pg.clone()
        pg_h[:, 0] = hid
        b = eng.forward(pg_h, poses, dims, tau).cpu().numpy().astype(np.float64)
        eng.check()
        print("cube hull vs box primitive", errors(a, b))
        assert np.abs(a - b).max() <= 2e-6
        check_forward(a, wb, eng.params(), what="box primitive")
    finally:
        eng.close()
