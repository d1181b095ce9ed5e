"""Pins of the oracle's superquadric union SDF and of sphere tracing (Sec. IV-B, IV-B1;
Supplement, mesh-SDF discrepancies)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle.edge_edge import ee_candidates, trace_to_surface
from oracle.manifold import Params, pair_manifold
from oracle.sdf import ELLIPSOID, SQ_UNION, quat_to_rot, sdf_local, sq_primitive

F64 = torch.float64
TAU = 1e-2


def t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


def prim_rows(prims):
    """Primitive rows in the geometry layout: (q), (t, eps1), (scale, eps2)."""
    rows = []
    for q, c, sc, e1, e2 in prims:
        q = np.asarray(q, np.float64) / np.linalg.norm(q)
        rows += [list(q), [c[0], c[1], c[2], e1], [sc[0], sc[1], sc[2], e2]]
    return t(rows)


def union_sdf(prims, y, tau=TAU):
    return sdf_local(SQ_UNION, y, torch.ones(3, dtype=F64), prim_rows(prims), tau)


I = [1.0, 0.0, 0.0, 0.0]


def test_single_unit_exponent_primitive_is_the_ellipsoid():
    rng = np.random.default_rng(0)
    dims = np.array([0.3, 0.5, 0.7])
    y = t(rng.normal(size=(200, 3)))
    phi, n = union_sdf([(I, [0, 0, 0], dims, 1.0, 1.0)], y)
    phi_e, n_e = sdf_local(ELLIPSOID, y, t(dims), None, TAU)
    assert torch.allclose(phi, phi_e, atol=1e-12, rtol=0)
    assert torch.allclose(n, n_e, atol=1e-12, rtol=0)


def test_sphere_closed_form():
    y = t(np.random.default_rng(1).normal(size=(100, 3)))
    phi, _ = union_sdf([(I, [0, 0, 0], [0.4, 0.4, 0.4], 1.0, 1.0)], y)
    assert torch.allclose(phi, y.norm(dim=1) - 0.4, atol=1e-12, rtol=0)


@pytest.mark.parametrize("e1,e2", [(0.3, 1.5), (1.5, 0.3), (0.7, 0.7), (1.9, 0.1), (0.1, 1.9)])
def test_zero_on_parametric_surface(e1, e2):
    """Points of the superellipsoid parametrisation (synth's mesh generator, not the
    implicit function) lie on the zero set, for exponents that tell eps1 from eps2."""
    sc = (0.3, 0.45, 0.6)
    pts, _ = synth.superellipsoid_surface(6, 12, sc, e1, e2)
    phi, gf = sq_primitive(t(pts), t(sc), e1, e2)
    assert phi.abs().max() < 1e-12
    # on an axis-free surface point a swapped exponent must miss the surface
    if e1 != e2:
        phi_sw, _ = sq_primitive(t(pts), t(sc), e2, e1)
        assert phi_sw.abs().max() > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_closed_form(axis):
    """On a principal axis f is (s)^(2/eps1) at s times the semi-axis, so
    phi = (1 - 1/s) s a = (s - 1) a for any exponents."""
    sc = np.array([0.3, 0.45, 0.6])
    s = np.array([0.3, 0.8, 1.0, 1.7, 3.0])
    y = np.zeros((len(s), 3))
    y[:, axis] = s * sc[axis]
    phi, _ = sq_primitive(t(y), t(sc), 0.4, 1.3)
    assert np.allclose(phi.numpy(), (s - 1.0) * sc[axis], atol=1e-12)


def test_grad_f_matches_finite_differences():
    rng = np.random.default_rng(2)
    sc, e1, e2 = t([0.3, 0.45, 0.6]), 0.6, 1.4
    x = t(rng.normal(size=(50, 3)) * 0.5)

    def f_of(x):  # the implicit function itself, written out on its own
        xt = (x / sc).abs()
        return (xt[:, 0] ** (2 / e2) + xt[:, 1] ** (2 / e2)) ** (e2 / e1) + xt[:, 2] ** (2 / e1)
    _, g = sq_primitive(x, sc, e1, e2)
    h = 1e-6
    fd = torch.stack([(f_of(x + h * torch.eye(3, dtype=F64)[i]) - f_of(x - h * torch.eye(3, dtype=F64)[i])) / (2 * h)
                      for i in range(3)], dim=1)
    assert torch.allclose(g, fd, rtol=1e-6, atol=1e-6)


def test_normal_parallel_to_grad_phi_on_the_surface():
    """f = 1 is phi = 0, so on the surface grad f and grad phi are parallel."""
    sc, e1, e2 = (0.3, 0.45, 0.6), 0.6, 1.4
    pts, _ = synth.superellipsoid_surface(4, 8, sc, e1, e2)
    pts = pts[np.abs(pts).min(1) > 1e-3]            # away from the axes
    x = t(pts).requires_grad_(True)
    phi, g = sq_primitive(x, t(sc), e1, e2)
    gphi, = torch.autograd.grad(phi.sum(), x)
    cos = (g * gphi).sum(1) / (g.norm(dim=1) * gphi.norm(dim=1))
    assert (cos > 1 - 1e-10).all()


def test_union_bounds_and_hard_limit():
    rng = np.random.default_rng(3)
    prims = [(synth.random_quaternions(rng, 1)[0], rng.uniform(-0.3, 0.3, 3), rng.uniform(0.1, 0.3, 3),
              *rng.uniform(0.3, 1.5, 2)) for _ in range(5)]
    y = t(rng.normal(size=(300, 3)) * 0.6)
    P = prim_rows(prims).reshape(-1, 3, 4)
    phis = []
    for l in range(5):
        R = quat_to_rot(P[l, 0])
        ph, _ = sq_primitive((y - P[l, 1, :3]) @ R, P[l, 2, :3], P[l, 1, 3], P[l, 2, 3])
        phis.append(ph)
    m = torch.stack(phis, 1).min(1).values
    phi, _ = union_sdf(prims, y)
    assert (phi <= m + 1e-12).all() and (phi >= m - TAU * math.log(5) - 1e-12).all()
    phi0, _ = union_sdf(prims, y, tau=1e-6)
    assert torch.allclose(phi0, m, atol=1e-5 * math.log(5) + 1e-12, rtol=0)


def test_duplicated_primitive_closed_form():
    """L copies of one primitive: phi = phi_1 - tau ln L, the normal unchanged."""
    pr = ([0.9, 0.1, -0.3, 0.2], [0.1, -0.2, 0.05], [0.3, 0.2, 0.4], 0.5, 1.2)
    y = t(np.random.default_rng(4).normal(size=(50, 3)) * 0.5)
    p1, n1 = union_sdf([pr], y)
    p3, n3 = union_sdf([pr] * 3, y)
    assert torch.allclose(p3, p1 - TAU * math.log(3), atol=1e-12, rtol=0)
    assert torch.allclose(n3, n1, atol=1e-12, rtol=0)


def test_frame_invariance():
    """Moving a primitive and the query point together leaves phi unchanged and rotates
    the normal with them."""
    rng = np.random.default_rng(5)
    q = synth.random_quaternions(rng, 1)[0]
    c = np.array([0.2, -0.1, 0.3])
    y0 = rng.normal(size=(40, 3)) * 0.4
    R = quat_to_rot(t(q))
    phi0, n0 = union_sdf([(I, [0, 0, 0], [0.3, 0.2, 0.4], 0.5, 1.2)], t(y0))
    phi1, n1 = union_sdf([(q, c, [0.3, 0.2, 0.4], 0.5, 1.2)], t(y0) @ R.T + t(c))
    assert torch.allclose(phi0, phi1, atol=1e-12, rtol=0)
    assert torch.allclose(n0 @ R.T, n1, atol=1e-12, rtol=0)


def test_trace_sphere_one_step_exact():
    """For a metric SDF (a sphere) one step along grad phi lands on the surface."""
    y = t(np.random.default_rng(6).normal(size=(30, 3)))
    sdf = lambda x: union_sdf([(I, [0, 0, 0], [0.4, 0.4, 0.4], 1.0, 1.0)], x)
    x1 = trace_to_surface(y, sdf, 1)
    assert torch.allclose(x1, 0.4 * y / y.norm(dim=1, keepdim=True), atol=1e-12, rtol=0)
    x3 = trace_to_surface(y, sdf, 3)
    assert torch.allclose(x3, x1, atol=1e-12, rtol=0)


def test_trace_converges_on_a_superquadric():
    """Near the surface of a boxy superquadric the fixed-direction iteration contracts
    towards the zero set step by step (phi measures the distance along the ray from the
    centre, not along the step, so one step is not enough and convergence is linear)."""
    pr = (I, [0, 0, 0], [0.3, 0.45, 0.6], 0.4, 1.3)
    pts, _ = synth.superellipsoid_surface(4, 8, pr[2], pr[3], pr[4])
    y = t(pts * 1.05 + np.random.default_rng(7).normal(size=pts.shape) * 0.01)
    sdf = lambda x: union_sdf([pr], x, tau=1e-4)
    res = [sdf(trace_to_surface(y, sdf, k))[0].abs().max().item() if k else sdf(y)[0].abs().max().item()
           for k in range(6)]
    assert all(b < 0.5 * a for a, b in zip(res, res[1:]))


def test_trace_off_changes_nothing_and_on_moves_only_points_and_geometry_terms():
    box = synth.primitive_geometry(synth.KIND_BOX)
    w = synth.config_box_box(n=2)
    pose, dims = t(w.poses[0]), t(w.dims[0])
    m0 = pair_manifold(box, box, pose, dims, TAU, Params())
    m0b = pair_manifold(box, box, pose, dims, TAU, Params(trace_iters=0))
    assert torch.equal(m0, m0b)
    # tracing onto a box whose mesh lies on its SDF surface moves the witnesses little
    m2 = pair_manifold(box, box, pose, dims, TAU, Params(trace_iters=2))
    assert (m2 - m0).abs().max() < 0.05


def test_union_body_vertices_near_zero_set():
    """The synthetic union meshes keep only vertices on the body's surface: each lies on
    its own primitive's zero set, and the smooth union moves phi by at most tau ln L."""
    rng = np.random.default_rng(8)
    g = synth.random_sq_union(rng, 5)
    phi, _ = sdf_local(SQ_UNION, t(g.verts[:, :3]), torch.ones(3, dtype=F64), t(g.planes), TAU)
    assert phi.max() < 1e-6           # vertices and primitives are stored in FP32
    assert (phi > -TAU * math.log(5) - 0.02).double().mean() > 0.9


@pytest.mark.parametrize("trace", [0, 3])
def test_one_primitive_union_body_equals_ellipsoid_body(trace):
    """A body given as a union of one eps = 1 superquadric with the ellipsoid's own mesh
    produces the same manifold against a box as the ellipsoid kind itself."""
    dims = np.array([0.35, 0.5, 0.25])
    ell = synth.primitive_geometry(synth.KIND_ELLIPSOID)
    verts = ell.verts.copy()
    verts[:, :3] *= dims
    planes = np.array([[1, 0, 0, 0], [0, 0, 0, 1.0], [dims[0], dims[1], dims[2], 1.0]], np.float32)
    sq = synth.Geometry(synth.KIND_SQ_UNION, np.ones(3, np.float32), verts, ell.edges.copy(), planes)
    box = synth.primitive_geometry(synth.KIND_BOX)
    rng = np.random.default_rng(9)
    q = synth.random_quaternions(rng, 2)
    pose = t(np.concatenate([q[0], [0, 0, 0], q[1], [0.1, 0.0, 0.62]]))
    prm = Params(trace_iters=trace)
    m_ell = pair_manifold(ell, box, pose, t(np.concatenate([dims, [0.3, 0.3, 0.3]])), TAU, prm)
    m_sq = pair_manifold(sq, box, pose, t([1, 1, 1, 0.3, 0.3, 0.3]), TAU, prm)
    assert torch.allclose(m_ell, m_sq, atol=1e-6, rtol=0)
