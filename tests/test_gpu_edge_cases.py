"""Edge cases of the manifold on the GPU against the oracle: the largest geometry the
library accepts, exactly parallel and coincident configurations, a ragged batch."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _parity import check_forward, check_grad, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    from paper_2602_20304_gb300.engine import Engine
    e = Engine(0)
    yield e
    e.close()


def run(engine, w, grad_out=None, **pkw):
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params(**pkw)
    out = engine.forward(pg, poses, dims, tau, params).cpu().numpy().astype(np.float64)
    grads = None
    if grad_out is not None:
        gp, gd = engine.backward(pg, poses, dims, tau, torch.as_tensor(grad_out, dtype=torch.float32,
                                                                      device="cuda"), params)
        grads = (gp.cpu().numpy().astype(np.float64), gd.cpu().numpy().astype(np.float64))
    torch.cuda.synchronize()
    engine.check()
    return out, grads, params


def make_workload(geoms, pair_geoms, poses, dims, tau):
    return synth.Workload("edge", geoms, np.asarray(pair_geoms, np.int32), np.asarray(poses, np.float32),
                          np.asarray(dims, np.float32), np.asarray(tau, np.float32))


def sphere_hull(n, seed):
    u = np.random.default_rng(seed).normal(size=(n, 3))
    return synth.hull_from_points(u / np.linalg.norm(u, axis=1, keepdims=True))


def test_largest_geometry_forward_and_adjoint(engine):
    """A 256-vertex hull (762 edges, 508 planes) against a capsule (144 edges)."""
    big = sphere_hull(256, 0)
    assert (big.n_verts, big.n_edges, big.n_planes) == (256, 762, 508)
    cap = synth.primitive_geometry(synth.KIND_CAPSULE)
    rng = np.random.default_rng(1)
    q = synth.random_quaternions(rng, 2)
    poses = [np.concatenate([q[0], [0, 0, 0], q[1], [0.0, 0.0, 1.25]])]
    dims = [[1, 1, 1, 0.3, 0.4, 0]]
    w = make_workload([big, cap], [[0, 1]], poses, dims, [1e-2])
    g = rng.normal(size=(1, 8, 8))
    out, (gp, gd), params = run(engine, w, grad_out=g)
    check_forward(out, w, params, what="largest geometry")
    check_grad(np.concatenate([gp, gd], 1), w, params, g, what="largest geometry gradients")


def qz(a):
    return [np.cos(a / 2), 0, 0, np.sin(a / 2)]


def test_exactly_parallel_edges(engine):
    """Boxes of different sizes, axis-aligned or turned about z only, so that many E-E pairs
    have exactly parallel edges (the QP's Q^T Q is singular without the L2 term): forward and
    adjoint against the oracle."""
    box = synth.primitive_geometry(synth.KIND_BOX)
    I = [1, 0, 0, 0]
    poses = [I + [0, 0, 0] + I + [0.31, 0.17, 0.51],
             I + [0, 0, 0] + qz(0.3) + [0.23, -0.12, 0.52],
             I + [0.02, 0.01, 0] + I + [0.55, 0.41, 0.25]]
    dims = [[0.5, 0.4, 0.3, 0.35, 0.45, 0.25]] * 2 + [[0.5, 0.4, 0.3, 0.3, 0.2, 0.3]]
    w = make_workload([box], [[0, 0]] * 3, poses, dims, [1e-2] * 3)
    g = np.random.default_rng(2).normal(size=(3, 8, 8))
    out, (gp, gd), params = run(engine, w, grad_out=g)
    check_forward(out, w, params, what="parallel edges")
    check_grad(np.concatenate([gp, gd], 1), w, params, g, what="parallel edges gradients")


def test_symmetric_configurations(engine):
    """Two identical boxes resting, offset, and at the same pose.  The configuration is
    symmetric under swapping the bodies, so candidate scores tie exactly; SoftSort's sort and
    |s_(k) - s_j| are not differentiable at a tie and the gradient there is not unique.  The
    manifold is, and so is its derivative under a common translation of both bodies (every
    point moves with it, depths, normals and weights do not), which is checked instead."""
    box = synth.primitive_geometry(synth.KIND_BOX)
    I = [1, 0, 0, 0]
    poses = [I + [0, 0, 0] + I + [0, 0, 0.95],
             I + [0, 0, 0] + I + [0.3, 0.2, 0.9],
             I + [0.1, -0.2, 0.3] + I + [0.1, -0.2, 0.3]]
    dims = [[0.5] * 6] * 3
    w = make_workload([box], [[0, 0]] * 3, poses, dims, [1e-2] * 3)
    g = np.random.default_rng(3).normal(size=(3, 8, 8))
    out, (gp, gd), params = run(engine, w, grad_out=g)
    check_forward(out, w, params, what="symmetric boxes")
    assert np.isfinite(gp).all() and np.isfinite(gd).all()
    common = gp[:, 4:7] + gp[:, 11:14]
    expect = g[:, :, 0:3].sum(1)
    assert np.abs(common - expect).max() <= 1e-3 * np.abs(gp).max()


def test_ragged_batch_of_tiny_and_large_pairs(engine):
    """Tetrahedra (4 vertices, 6 edges) and the largest hulls in one batch."""
    tet = synth.hull_from_points(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) - 0.25)
    big = sphere_hull(200, 3)
    ell = synth.primitive_geometry(synth.KIND_ELLIPSOID)
    rng = np.random.default_rng(4)
    n = 9
    pg = [[i % 2, 2] for i in range(n)]                    # tet or big hull against an ellipsoid
    q = synth.random_quaternions(rng, 2 * n)
    poses = [np.concatenate([q[2 * i], rng.uniform(-0.1, 0.1, 3), q[2 * i + 1], [0, 0, 0.9]]) for i in range(n)]
    dims = [[1, 1, 1, 0.4, 0.5, 0.6]] * n
    w = make_workload([tet, big, ell], pg, poses, dims, [1e-2] * n)
    out, _, params = run(engine, w)
    check_forward(out, w, params, what="ragged batch")


def test_separated_bodies(engine):
    """Bodies far apart: every weight underflows and every score ties at zero, so each row is
    the plain average of all candidates (forward only; the gradient is not unique there)."""
    hull = sphere_hull(40, 5)
    cyl = synth.primitive_geometry(synth.KIND_CYLINDER)
    rng = np.random.default_rng(6)
    q = synth.random_quaternions(rng, 4)
    poses = [np.concatenate([q[0], [0, 0, 0], q[1], [0, 0, 3.0]]),
             np.concatenate([q[2], [0, 0, 0], q[3], [2.5, 1.0, 0]])]
    dims = [[1, 1, 1, 0.4, 0.4, 0.5]] * 2
    w = make_workload([hull, cyl], [[0, 1]] * 2, poses, dims, [1e-2, 1e-1])
    out, _, params = run(engine, w)
    check_forward(out, w, params, what="separated bodies")
