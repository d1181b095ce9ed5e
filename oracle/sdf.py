"""Smooth SDF primitives and their contact normals (Sec. IV-B; Sec. IV-C).

Test infrastructure (see ``oracle/__init__``).  Shapes are in their local
frame; a body with pose (q, t) maps local y to world R(q / |q|) y + t.

Primitive definitions (tau is the smoothing of the pair):

* box, half-extents h: convex polyhedron of the 6 planes +-e_i . y - h_i;
  phi = LSE_tau of the plane values (Sec. IV-B2).
* hull: the same LSE over its outward face planes n_f . y - o_f (Sec. IV-B2).
* ellipsoid (a, b, c): superquadric with eps1 = eps2 = 1, f = |y~|^2 with
  y~ = (y_x / a, y_y / b, y_z / c), phi = (1 - f^(-1/2)) |y| (Sec. IV-B1; the
  printed "/ |x|" is read as a product, which makes a sphere's phi exactly
  |y| - r).  Its normal is built from grad f, as the footnote of Sec. IV-C
  prescribes for superquadrics.
* capsule (r, h) along z: phi = |y - clip_s(y_z, -h, h, tau) z| - r (reading,
  not a paper primitive; tends to the exact capsule SDF as tau -> 0).
* cylinder (r, h) along z: phi = LSE_tau(rho - r, y_z - h, -y_z - h) with
  rho = sqrt(y_x^2 + y_y^2) (reading, convex-polyhedron style).
* union of superquadrics (Sec. IV-B): primitive l has an orientation R_l and
  centre t_l in the body frame, axis lengths (a, b, c) and exponents
  (eps1, eps2).  At x = R_l^T (y - t_l) and x~ = (x_x / a, x_y / b, x_z / c),
  f_l = ((x~_x^2)^(1/eps2) + (x~_y^2)^(1/eps2))^(eps2/eps1) + (x~_z^2)^(1/eps1)
  and phi_l = (1 - f_l^(-eps1/2)) |x| (Sec. IV-B1, the printed "/ |x|" read as
  a product as for the ellipsoid); the body is their smooth union
  phi = -LSE_tau(-phi_1, ..., -phi_L) (Sec. IV-B, temperature tau: reading).
  The normal uses grad f as for every superquadric (Sec. IV-C footnote); for a
  union the primitives' gradients R_l grad_x f_l are blended with the union's
  own weights softmax(-phi_l / tau), i.e. as d phi / d phi_l (reading: the
  paper gives no union normal).  A single primitive with eps1 = eps2 = 1 is
  the ellipsoid above.

Normal of every primitive: g / sqrt(tau + |g|^2) with g = grad phi (grad f for
the ellipsoid), the regularised form the paper gives for all three families.

Pins: tests/test_oracle_sdf.py -- cube centre and face-centre closed forms,
sphere = |y| - r exactly, tau -> 0 limits against the exact box, capsule and
cylinder distances, LSE bounds for hulls, and the explicit gradients against
central finite differences of phi.  Superquadric unions:
tests/test_oracle_sq_union.py -- the single eps = 1 primitive equals the
ellipsoid, phi = 0 on parametric surface points for any exponents, the axis
closed form phi = (s - 1) a at s a on an axis, union bounds and the duplicated
primitive closed form, frame invariance, grad f against finite differences.
"""
import torch

from .smooth import clip_s, lse, sigmoid

BOX, CAPSULE, CYLINDER, ELLIPSOID, HULL, SQ_UNION = 0, 1, 2, 3, 4, 5


def quat_to_rot(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z)."""
    q = q / torch.linalg.vector_norm(q)
    w, x, y, z = q[0], q[1], q[2], q[3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)])])


def local_vertices(kind, template, dims):
    """Mesh vertices in the local frame from the template rows (u_x, u_y, u_z, s)."""
    u, s = template[:, :3], template[:, 3]
    if kind in (BOX, ELLIPSOID):
        return u * dims
    if kind == CYLINDER:
        return torch.stack([dims[0] * u[:, 0], dims[0] * u[:, 1], dims[1] * u[:, 2]], dim=1)
    if kind == CAPSULE:
        return torch.stack([dims[0] * u[:, 0], dims[0] * u[:, 1],
                            dims[0] * u[:, 2] + s * dims[1]], dim=1)
    if kind in (HULL, SQ_UNION):
        return u.clone()
    raise ValueError(kind)


def _safe_norm(v):
    r2 = (v * v).sum(-1)
    pos = r2 > 0
    r = torch.sqrt(torch.where(pos, r2, torch.ones_like(r2)))
    return torch.where(pos, r, torch.zeros_like(r))


def _planes_of(kind, dims, planes):
    """(normals (F, 3), offsets (F,)) of a convex-polyhedron primitive."""
    if kind == BOX:
        eye = torch.eye(3, dtype=dims.dtype)
        n = torch.cat([eye, -eye], dim=0)
        o = torch.cat([dims, dims])
        return n, o
    return planes[:, :3], planes[:, 3]


def _normalise(g, tau):
    return g / torch.sqrt(tau + (g * g).sum(-1, keepdim=True))


_TINY = 1e-300


def sq_primitive(x, scale, eps1, eps2):
    """(phi, grad f) of one superquadric at points ``x`` (..., 3) of its own frame."""
    xt = x / scale
    ax = torch.abs(xt).clamp_min(_TINY)
    p1, p2, r = 2.0 / eps1, 2.0 / eps2, eps2 / eps1
    u = ax[..., 0] ** p2
    v = ax[..., 1] ** p2
    w = ax[..., 2] ** p1
    suv = (u + v).clamp_min(_TINY)
    f = suv ** r + w
    phi = (1.0 - f.clamp_min(_TINY) ** (-0.5 * eps1)) * _safe_norm(x)
    ds = r * suv ** (r - 1.0)
    sg = torch.sign(xt)
    gx = ds * p2 * ax[..., 0] ** (p2 - 1.0) * sg[..., 0]
    gy = ds * p2 * ax[..., 1] ** (p2 - 1.0) * sg[..., 1]
    gz = p1 * ax[..., 2] ** (p1 - 1.0) * sg[..., 2]
    return phi, torch.stack([gx, gy, gz], dim=-1) / scale


def sq_union_parts(y, prims, tau):
    """(phi, grad for the normal) of a union of superquadrics at body-frame points y."""
    P = prims.reshape(-1, 3, 4)
    phis, grads = [], []
    for l in range(P.shape[0]):
        R = quat_to_rot(P[l, 0])
        x = (y - P[l, 1, :3]) @ R                      # R^T (y - t) for row vectors
        ph, g = sq_primitive(x, P[l, 2, :3], P[l, 1, 3], P[l, 2, 3])
        phis.append(ph)
        grads.append(g @ R.T)
    phis = torch.stack(phis, dim=-1)                   # (..., L)
    grads = torch.stack(grads, dim=-2)                 # (..., L, 3)
    phi = -lse(-phis, tau, dim=-1)
    pi = torch.softmax(-phis / tau, dim=-1)
    return phi, (pi[..., None] * grads).sum(-2)


def sdf_local(kind, y, dims, planes, tau):
    """(phi, normal) at local points ``y`` (..., 3).  See the module header."""
    if kind in (BOX, HULL):
        n, o = _planes_of(kind, dims, planes)
        s = y @ n.T - o                                  # (..., F) plane values
        phi = lse(s, tau, dim=-1)
        pi = torch.softmax(s / tau, dim=-1)              # d LSE / d s
        g = pi @ n
        return phi, _normalise(g, tau)
    if kind == ELLIPSOID:
        yt = y / dims
        f = (yt * yt).sum(-1)
        r = _safe_norm(y)
        phi = r * (1.0 - f.rsqrt())
        gf = 2.0 * y / (dims * dims)
        return phi, _normalise(gf, tau)
    if kind == CAPSULE:
        rad, h = dims[0], dims[1]
        c = clip_s(y[..., 2], -h, h, tau)
        w = torch.stack([y[..., 0], y[..., 1], y[..., 2] - c], dim=-1)
        r = _safe_norm(w)
        phi = r - rad
        dc = sigmoid((y[..., 2] + h) / tau) - sigmoid((y[..., 2] - h) / tau)
        rs = torch.where(r > 0, r, torch.ones_like(r))
        g = torch.stack([w[..., 0], w[..., 1], w[..., 2] * (1.0 - dc)], dim=-1) / rs[..., None]
        g = torch.where((r > 0)[..., None], g, torch.zeros_like(g))
        return phi, _normalise(g, tau)
    if kind == CYLINDER:
        rad, h = dims[0], dims[1]
        rho = _safe_norm(y[..., :2])
        s = torch.stack([rho - rad, y[..., 2] - h, -y[..., 2] - h], dim=-1)
        phi = lse(s, tau, dim=-1)
        pi = torch.softmax(s / tau, dim=-1)
        rhos = torch.where(rho > 0, rho, torch.ones_like(rho))
        radial = torch.where((rho > 0)[..., None], y[..., :2] / rhos[..., None],
                             torch.zeros_like(y[..., :2]))
        g = torch.stack([pi[..., 0] * radial[..., 0], pi[..., 0] * radial[..., 1],
                         pi[..., 1] - pi[..., 2]], dim=-1)
        return phi, _normalise(g, tau)
    if kind == SQ_UNION:
        phi, g = sq_union_parts(y, planes, tau)
        return phi, _normalise(g, tau)
    raise ValueError(kind)


def sdf_world(kind, x, R, t, dims, planes, tau):
    """(phi, world normal) of a posed body at world points ``x`` (..., 3)."""
    y = (x - t) @ R                                      # R^T (x - t) for row vectors
    phi, nu = sdf_local(kind, y, dims, planes, tau)
    return phi, nu @ R.T
