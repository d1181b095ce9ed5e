"""Bodies made of superquadrics (smooth union, general exponents) and sphere-traced E-E
witnesses on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import synth
from _parity import check_forward, check_grad

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


@pytest.mark.parametrize("n_prims", [1, 5])
def test_union_full_manifold(engine, n_prims):
    """Every vertex and every edge pair of two multi-superquadric bodies."""
    w = synth.config_sq_union(n=16, n_prims=n_prims, pool=4, seed=synth.SEED_BASE + 60 + n_prims)
    gpu, params = run(engine, w)
    check_forward(gpu, w, params, what=f"sq union L={n_prims}")


def test_union_with_one_edge_per_primitive(engine):
    """The paper's armadillo setting with synthetic primitives: 18 superquadrics per body,
    all vertices, the 18 deepest soft edges per body."""
    w = synth.config_sq_union(n=24, n_prims=18, pool=6)
    gpu, params = run(engine, w, top_edges=18)
    check_forward(gpu, w, params, what="sq union 18, top 18 edges")


@pytest.mark.parametrize("cfg,n,kw", [(1, 32, {}), (2, 24, {}), ("sq", 16, dict(top_edges=5))])
@pytest.mark.parametrize("iters", [1, 3])
def test_sphere_traced_witnesses(engine, cfg, n, kw, iters):
    w = synth.config_sq_union(n=n, n_prims=5, pool=4) if cfg == "sq" else synth.make_config(cfg, n)
    gpu, params = run(engine, w, trace_iters=iters, **kw)
    check_forward(gpu, w, params, what=f"trace {iters} on {cfg}")


def test_one_unit_exponent_primitive_equals_the_ellipsoid_kind(engine):
    """The union kind with one eps = 1 superquadric and the ellipsoid's mesh reproduces the
    ellipsoid kind against the same partners, in the same launch."""
    rng = np.random.default_rng(11)
    dims = np.array([0.35, 0.5, 0.25], np.float32)
    ell = synth.primitive_geometry(synth.KIND_ELLIPSOID, dims)
    verts = ell.verts.copy()
    verts[:, :3] *= dims
    planes = np.array([[1, 0, 0, 0], [0, 0, 0, 1.0], [dims[0], dims[1], dims[2], 1.0]], np.float32)
    sq = synth.Geometry(synth.KIND_SQ_UNION, np.ones(3, np.float32), verts, ell.edges.copy(), planes)
    hull = synth.hull_from_points(rng.normal(size=(30, 3)) * 0.4)
    n = 32
    q = synth.random_quaternions(rng, 2 * n)
    poses = np.concatenate([q[:n], rng.uniform(-0.05, 0.05, (n, 3)), q[n:], np.tile([0, 0, 0.5], (n, 1))], 1)
    w_ell = synth.Workload("ell", [ell, hull], np.tile([0, 1], (n, 1)).astype(np.int32), poses.astype(np.float32),
                           np.tile(np.concatenate([dims, [1, 1, 1]]), (n, 1)).astype(np.float32),
                           np.full(n, 1e-2, np.float32))
    w_sq = synth.Workload("sq", [sq, hull], w_ell.pair_geoms, w_ell.poses, np.ones((n, 6), np.float32), w_ell.tau)
    a, _ = run(engine, w_ell)
    b, _ = run(engine, w_sq)
    assert np.abs(a - b).max() < 2e-5


@pytest.mark.parametrize("n_prims,n", [(1, 8), (3, 8), (5, 4)])
def test_union_adjoint_matches_oracle_autograd(engine, n_prims, n):
    """dL/d poses of multi-superquadric pairs (every vertex and edge pair) against the
    FP64 oracle's autograd under the per-pair bar (1e-3 of each pair's largest component)."""
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.config_sq_union(n=n, n_prims=n_prims, pool=3, seed=synth.SEED_BASE + 70 + n_prims)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params()
    g = np.random.default_rng(n_prims).normal(size=(n, 8, 8))
    gp, gd = engine.backward(pg, poses, dims, tau, torch.as_tensor(g, dtype=torch.float32, device="cuda"), params)
    torch.cuda.synchronize()
    engine.check()
    got = np.concatenate([gp.cpu().numpy(), gd.cpu().numpy()], 1).astype(np.float64)
    check_grad(got, w, params, g, what=f"sq union L={n_prims} gradients")
    assert np.abs(gd.cpu().numpy()).max() == 0.0     # dims are unused by the union kind


@pytest.mark.parametrize("cfg,n", [(1, 16), (2, 12), ("sq", 6)])
@pytest.mark.parametrize("iters", [1, 3])
def test_traced_adjoint_matches_oracle_autograd(engine, cfg, n, iters):
    """The adjoint through sphere tracing (fixed direction from the SDF gradient at the QP
    witness, unrolled steps) against the oracle's autograd."""
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.config_sq_union(n=n, n_prims=3, pool=3) if cfg == "sq" else synth.make_config(cfg, n)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params(trace_iters=iters)
    g = np.random.default_rng(iters).normal(size=(n, 8, 8))
    gp, gd = engine.backward(pg, poses, dims, tau, torch.as_tensor(g, dtype=torch.float32, device="cuda"), params)
    torch.cuda.synchronize()
    engine.check()
    got = np.concatenate([gp.cpu().numpy(), gd.cpu().numpy()], 1).astype(np.float64)
    check_grad(got, w, params, g, what=f"trace {iters} on {cfg} gradients")
