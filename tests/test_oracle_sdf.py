"""Pins of the oracle's SDF primitives (Sec. IV-B) against closed forms and exact distances."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.sdf import BOX, CAPSULE, CYLINDER, ELLIPSOID, HULL, sdf_local

F = torch.float64
NO_PLANES = torch.zeros((0, 4), dtype=F)


def t(x):
    return torch.as_tensor(np.asarray(x), dtype=F)


def exact_box(y, h):
    q = np.abs(y) - h
    return np.linalg.norm(np.maximum(q, 0), axis=-1) + np.minimum(q.max(-1), 0)


def exact_capsule(y, r, h):
    z = np.clip(y[..., 2], -h, h)
    w = y.copy()
    w[..., 2] -= z
    return np.linalg.norm(w, axis=-1) - r


def exact_cylinder(y, r, h):
    d = np.stack([np.hypot(y[..., 0], y[..., 1]) - r, np.abs(y[..., 2]) - h], -1)
    return np.linalg.norm(np.maximum(d, 0), axis=-1) + np.minimum(d.max(-1), 0)


@pytest.mark.parametrize("h,tau", [(0.5, 1e-2), (0.3, 1e-1), (1.0, 1e-3)])
def test_cube_centre_closed_form(h, tau):
    # all six planes read -h at the centre: LSE = -h + tau ln 6
    phi, nu = sdf_local(BOX, t([[0.0, 0.0, 0.0]]), t([h, h, h]), NO_PLANES, tau)
    assert abs(phi.item() - (-h + tau * np.log(6))) < 1e-14
    assert nu.abs().max().item() < 1e-14          # symmetric: gradient vanishes


def test_box_tau_to_zero_inside_and_face_regions():
    rng = np.random.default_rng(1)
    h = np.array([0.5, 0.3, 0.8])
    y = rng.uniform(-1, 1, size=(400, 3)) * h          # inside
    face = np.zeros((200, 3))
    face[:, 0] = h[0] + rng.uniform(0, 0.3, 200)       # outside through the +x face
    face[:, 1] = rng.uniform(-h[1], h[1], 200)
    face[:, 2] = rng.uniform(-h[2], h[2], 200)
    pts = np.concatenate([y, face])
    phi, _ = sdf_local(BOX, t(pts), t(h), NO_PLANES, 1e-6)
    assert np.abs(phi.numpy() - exact_box(pts, h)).max() < 1e-5 * (1 + np.log(6))


def test_box_lse_brackets_exact_inside():
    rng = np.random.default_rng(2)
    h = np.array([0.4, 0.6, 0.5])
    y = rng.uniform(-1, 1, size=(300, 3)) * h
    for tau in (1e-2, 1e-1):
        phi, _ = sdf_local(BOX, t(y), t(h), NO_PLANES, tau)
        ex = exact_box(y, h)
        assert (phi.numpy() >= ex - 1e-12).all()
        assert (phi.numpy() <= ex + tau * np.log(6) + 1e-12).all()


@pytest.mark.parametrize("tau", [1e-3, 1e-2, 1e-1])
def test_sphere_is_exact(tau):
    rng = np.random.default_rng(3)
    r = 0.7
    y = rng.normal(size=(500, 3)) * 0.8
    phi, nu = sdf_local(ELLIPSOID, t(y), t([r, r, r]), NO_PLANES, tau)
    assert np.abs(phi.numpy() - (np.linalg.norm(y, axis=1) - r)).max() < 1e-13
    # normal parallel to y
    cos = (nu.numpy() * y).sum(1) / np.linalg.norm(nu.numpy(), axis=1) / np.linalg.norm(y, axis=1)
    assert np.abs(cos - 1).max() < 1e-12


def test_ellipsoid_zero_set_and_sign():
    rng = np.random.default_rng(4)
    d = np.array([0.3, 0.9, 0.5])
    u = rng.normal(size=(200, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    surf = u * d
    phi, _ = sdf_local(ELLIPSOID, t(surf), t(d), NO_PLANES, 1e-2)
    assert np.abs(phi.numpy()).max() < 1e-13
    inside, _ = sdf_local(ELLIPSOID, t(surf * 0.8), t(d), NO_PLANES, 1e-2)
    outside, _ = sdf_local(ELLIPSOID, t(surf * 1.2), t(d), NO_PLANES, 1e-2)
    assert (inside < 0).all() and (outside > 0).all()


def test_capsule_tau_to_zero():
    rng = np.random.default_rng(5)
    r, h = 0.3, 0.6
    y = rng.uniform(-1.2, 1.2, size=(500, 3))
    y = y[np.hypot(y[:, 0], y[:, 1]) > 0.05]
    phi, _ = sdf_local(CAPSULE, t(y), t([r, h, 0.0]), NO_PLANES, 1e-7)
    assert np.abs(phi.numpy() - exact_capsule(y, r, h)).max() < 1e-6


def test_cylinder_tau_to_zero_side_and_cap_regions():
    rng = np.random.default_rng(6)
    r, h = 0.4, 0.7
    y = rng.uniform(-1.2, 1.2, size=(2000, 3))
    rho = np.hypot(y[:, 0], y[:, 1])
    keep = (rho <= r) | (np.abs(y[:, 2]) <= h)          # not in the outer rim-corner region
    y = y[keep & (rho > 0.01)]
    phi, _ = sdf_local(CYLINDER, t(y), t([r, h, 0.0]), NO_PLANES, 1e-7)
    assert np.abs(phi.numpy() - exact_cylinder(y, r, h)).max() < 1e-6


def _hull():
    rng = np.random.default_rng(7)
    g = rng.normal(size=(40, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return synth.hull_from_points(g * rng.random(40)[:, None] ** (1 / 3))


def test_hull_structure_and_lse_bounds():
    g = _hull()
    V, E, Fn = g.n_verts, g.n_edges, g.n_planes
    assert V - E + Fn == 2                                    # Euler, closed triangulated surface
    pl = g.planes.astype(np.float64)
    assert np.abs(np.linalg.norm(pl[:, :3], axis=1) - 1).max() < 1e-6
    vals = g.verts[:, :3].astype(np.float64) @ pl[:, :3].T - pl[:, 3]
    assert vals.max() < 1e-5                                  # every vertex inside every plane
    rng = np.random.default_rng(8)
    y = rng.uniform(-1.5, 1.5, size=(300, 3))
    for tau in (1e-3, 1e-2, 1e-1):
        phi, _ = sdf_local(HULL, t(y), t([1, 1, 1]), t(pl), tau)
        mx = (y @ pl[:, :3].T - pl[:, 3]).max(1)
        assert (phi.numpy() >= mx - 1e-12).all()
        assert (phi.numpy() <= mx + tau * np.log(Fn) + 1e-12).all()


CASES = [
    (BOX, [0.5, 0.3, 0.4]),
    (CAPSULE, [0.3, 0.5, 0.0]),
    (CYLINDER, [0.4, 0.6, 0.0]),
    (HULL, None),
]


@pytest.mark.parametrize("kind,dims", CASES)
@pytest.mark.parametrize("tau", [1e-2, 1e-1])
def test_normals_against_finite_differences(kind, dims, tau):
    """normal = g / sqrt(tau + |g|^2) with g the central-FD gradient of phi."""
    rng = np.random.default_rng(9)
    planes = NO_PLANES
    if kind == HULL:
        planes = t(_hull().planes)
        dims = [1, 1, 1]
    y = rng.uniform(-1.0, 1.0, size=(60, 3))
    y = y[np.hypot(y[:, 0], y[:, 1]) > 0.05]
    hstep = 1e-6
    g = np.zeros_like(y)
    for a in range(3):
        e = np.zeros(3)
        e[a] = hstep
        fp, _ = sdf_local(kind, t(y + e), t(dims), planes, tau)
        fm, _ = sdf_local(kind, t(y - e), t(dims), planes, tau)
        g[:, a] = (fp.numpy() - fm.numpy()) / (2 * hstep)
    _, nu = sdf_local(kind, t(y), t(dims), planes, tau)
    ref = g / np.sqrt(tau + (g * g).sum(1, keepdims=True))
    assert np.abs(nu.numpy() - ref).max() < 1e-6


def test_ellipsoid_normal_from_grad_f():
    """Superquadric normal uses grad f (footnote of Sec. IV-C), checked by FD of f."""
    rng = np.random.default_rng(10)
    d = np.array([0.3, 0.8, 0.5])
    tau = 1e-2
    y = rng.uniform(-1, 1, size=(50, 3))
    f = lambda p: ((p / d) ** 2).sum(-1)  # noqa: E731  (inside-outside function, eps1 = eps2 = 1)
    hstep = 1e-6
    g = np.stack([(f(y + hstep * e) - f(y - hstep * e)) / (2 * hstep) for e in np.eye(3)], 1)
    _, nu = sdf_local(ELLIPSOID, t(y), t(d), NO_PLANES, tau)
    ref = g / np.sqrt(tau + (g * g).sum(1, keepdims=True))
    assert np.abs(nu.numpy() - ref).max() < 1e-7


def test_world_frame_and_vertices_on_surface():
    """Posed SDF equals the local SDF of the pulled-back point; template vertices map onto
    the exact surface of each primitive."""
    rng = np.random.default_rng(11)
    q = t(synth.random_quaternions(rng, 1)[0])
    R = oracle.quat_to_rot(q)
    assert torch.allclose(R @ R.T, torch.eye(3, dtype=F), atol=1e-14)
    assert abs(torch.linalg.det(R).item() - 1) < 1e-14
    for kind, dims, exact in [(BOX, [0.5, 0.3, 0.4], lambda y, d: exact_box(y, d)),
                              (CAPSULE, [0.3, 0.5, 0], lambda y, d: exact_capsule(y, d[0], d[1])),
                              (CYLINDER, [0.4, 0.6, 0], lambda y, d: exact_cylinder(y, d[0], d[1]))]:
        geom = synth.primitive_geometry(kind)
        v = oracle.local_vertices(kind, t(geom.verts), t(dims)).numpy()
        assert np.abs(exact(v, np.array(dims))).max() < 1e-7
    tt = t([0.3, -0.2, 0.5])
    x = t(rng.normal(size=(20, 3)))
    phi_w, nu_w = oracle.sdf_world(BOX, x, R, tt, t([0.5, 0.3, 0.4]), NO_PLANES, 1e-2)
    phi_l, nu_l = sdf_local(BOX, (x - tt) @ R, t([0.5, 0.3, 0.4]), NO_PLANES, 1e-2)
    assert torch.allclose(phi_w, phi_l, atol=1e-15)
    assert torch.allclose(nu_w, nu_l @ R.T, atol=1e-15)
