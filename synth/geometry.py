"""Template meshes and convex hulls for the synthetic workloads.

A geometry carries the two representations the method attaches to every
surface (Sec. IV-A): a mesh (vertices and edges) and the parameters of a
smooth SDF primitive (Sec. IV-B).  For the four analytic primitives the mesh
is a *unit template*: each vertex row is ``(u_x, u_y, u_z, s)`` and the
library / oracle map it to a surface point from the primitive's dimensions
(box and ellipsoid scale each axis, cylinder and capsule scale the radius and
half-length).  For a convex hull the rows are the vertices themselves
(``s = 0``) and the SDF parameters are the outward face planes
``(n_x, n_y, n_z, o)``, with plane value ``n . y - o``.  A union of
superquadrics (Sec. IV-B, smooth union of SQ primitives) also carries its
vertices directly; its ``planes`` hold three rows per primitive:
``(q_w, q_x, q_y, q_z)`` (orientation in the body frame), ``(t_x, t_y, t_z,
eps1)`` and ``(a, b, c, eps2)`` (axis lengths and the two exponents).
"""
from __future__ import annotations

import dataclasses
import numpy as np

KIND_BOX, KIND_CAPSULE, KIND_CYLINDER, KIND_ELLIPSOID, KIND_HULL = 0, 1, 2, 3, 4
KIND_SQ_UNION = 5
KIND_NAMES = {KIND_BOX: "box", KIND_CAPSULE: "capsule", KIND_CYLINDER: "cylinder",
              KIND_ELLIPSOID: "ellipsoid", KIND_HULL: "hull", KIND_SQ_UNION: "sq_union"}


@dataclasses.dataclass
class Geometry:
    kind: int
    dims: np.ndarray          # (3,) float32, default dimensions
    verts: np.ndarray         # (V, 4) float32 template rows
    edges: np.ndarray         # (E, 2) int32 vertex indices
    planes: np.ndarray        # (F, 4) float32, hull only (else shape (0, 4))

    @property
    def n_verts(self):
        return int(self.verts.shape[0])

    @property
    def n_edges(self):
        return int(self.edges.shape[0])

    @property
    def n_planes(self):
        return int(self.planes.shape[0])


def _edges_from_faces(faces):
    es = set()
    for f in faces:
        m = len(f)
        for i in range(m):
            a, b = int(f[i]), int(f[(i + 1) % m])
            es.add((min(a, b), max(a, b)))
    return np.array(sorted(es), dtype=np.int32)


def box_template():
    """8 corners of the cube [-1, 1]^3 and its 12 edges."""
    v = np.array([[x, y, z, 0.0] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)],
                 dtype=np.float32)
    e = []
    for i in range(8):
        for j in range(i + 1, 8):
            if np.abs(v[i, :3] - v[j, :3]).sum() == 2.0:
                e.append((i, j))
    return v, np.array(e, dtype=np.int32)


def cylinder_template(n=16):
    """Two rings of ``n`` points on the unit cylinder rims (z = -1, +1)."""
    th = 2 * np.pi * np.arange(n) / n
    v = []
    for z in (-1.0, 1.0):
        for t in th:
            v.append((np.cos(t), np.sin(t), z, 0.0))
    e = []
    for r in range(2):
        for i in range(n):
            e.append((r * n + i, r * n + (i + 1) % n))
    for i in range(n):
        e.append((i, n + i))
    return np.array(v, dtype=np.float32), np.array(e, dtype=np.int32)


def capsule_template(n=16, lats=(0.0, np.pi / 4)):
    """Two hemispherical caps: rings at the given latitudes plus the poles.

    Row ``(u, s)`` maps to ``r * u + s * h * z_hat`` (s = +-1 picks the cap).
    """
    th = 2 * np.pi * np.arange(n) / n
    v, ring_ids = [], {}
    for s in (-1.0, 1.0):
        for li, lat in enumerate(lats):
            ids = []
            for t in th:
                ids.append(len(v))
                v.append((np.cos(lat) * np.cos(t), np.cos(lat) * np.sin(t), s * np.sin(lat), s))
            ring_ids[(s, li)] = ids
    poles = {}
    for s in (-1.0, 1.0):
        poles[s] = len(v)
        v.append((0.0, 0.0, s, s))
    e = []
    for key, ids in ring_ids.items():
        for i in range(n):
            e.append((ids[i], ids[(i + 1) % n]))
    for s in (-1.0, 1.0):
        for li in range(len(lats) - 1):
            a, b = ring_ids[(s, li)], ring_ids[(s, li + 1)]
            for i in range(n):
                e.append((a[i], b[i]))
        top = ring_ids[(s, len(lats) - 1)]
        for i in range(n):
            e.append((top[i], poles[s]))
    lo, hi = ring_ids[(-1.0, 0)], ring_ids[(1.0, 0)]
    for i in range(n):
        e.append((lo[i], hi[i]))
    e = np.array([(min(a, b), max(a, b)) for a, b in e], dtype=np.int32)
    return np.array(v, dtype=np.float32), e


def icosphere_template(level=1):
    """Subdivided icosahedron on the unit sphere (level 1: 42 vertices, 120 edges)."""
    t = (1.0 + 5 ** 0.5) / 2.0
    p = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    pts = [np.array(q, dtype=np.float64) / np.linalg.norm(q) for q in p]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache, nf = {}, []

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in cache:
                m = pts[a] + pts[b]
                pts.append(m / np.linalg.norm(m))
                cache[k] = len(pts) - 1
            return cache[k]
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    v = np.zeros((len(pts), 4), dtype=np.float32)
    v[:, :3] = np.array(pts)
    return v, _edges_from_faces(faces)


def hull_from_points(points, eps_rel=1e-9):
    """Convex hull of a point set: compact vertex list, unique edges, face planes.

    Uses qhull (scipy).  qhull reports triangles; neighbouring triangles whose planes
    agree within eps (eps_rel x the bounding-box diagonal) form one flat facet with
    one plane (a box face is one plane, not two), the edges inside a facet are
    dropped, and so are points left without an edge (in the middle of a facet).
    Each plane row is ``(n, o)`` with unit outward normal ``n`` and offset
    ``o = n . p``; vertices keep the order of their index in ``points``."""
    from scipy.spatial import ConvexHull
    pts = np.asarray(points, dtype=np.float64)
    h = ConvexHull(pts)
    eps = eps_rel * np.linalg.norm(pts.max(0) - pts.min(0))
    eq = h.equations                       # n . x + off <= 0 inside
    tri = h.simplices
    nt = len(tri)
    root = list(range(nt))

    def find(t):
        while root[t] != t:
            root[t] = root[root[t]]
            t = root[t]
        return t

    def coplanar(a, b):
        return (eq[a, :3] @ eq[b, :3] > 0 and np.abs(pts[tri[b]] @ eq[a, :3] + eq[a, 3]).max() <= eps
                and np.abs(pts[tri[a]] @ eq[b, :3] + eq[b, 3]).max() <= eps)
    for t in range(nt):
        for k in range(3):
            u = int(h.neighbors[t, k])
            if t < u and coplanar(t, u):
                root[find(t)] = find(u)
    es = set()
    for t in range(nt):
        for k in range(3):                 # the edge opposite vertex k borders neighbour k
            u = int(h.neighbors[t, k])
            if find(t) != find(u):
                a, b = int(tri[t, (k + 1) % 3]), int(tri[t, (k + 2) % 3])
                es.add((min(a, b), max(a, b)))
    vid = np.array(sorted({v for e in es for v in e}))
    remap = -np.ones(len(pts), dtype=np.int64)
    remap[vid] = np.arange(len(vid))
    edges = np.array(sorted((int(remap[a]), int(remap[b])) for a, b in es), dtype=np.int32)
    verts = np.zeros((len(vid), 4), dtype=np.float32)
    verts[:, :3] = pts[vid]
    facets = {}
    for t in range(nt):
        facets.setdefault(find(t), []).append(t)
    planes = np.zeros((len(facets), 4), dtype=np.float32)
    for j, ts in enumerate(facets.values()):
        area = np.zeros(3)
        for t in ts:                       # qhull's triangles are unoriented: orient each outward
            c = np.cross(pts[tri[t, 1]] - pts[tri[t, 0]], pts[tri[t, 2]] - pts[tri[t, 0]])
            area += c * np.sign(c @ eq[t, :3])
        n = area / np.linalg.norm(area)
        planes[j, :3] = n
        planes[j, 3] = np.mean([pts[tri[t]] @ n for t in ts])
    return Geometry(KIND_HULL, np.ones(3, dtype=np.float32), verts, edges, planes)


_TEMPLATES = {}


def primitive_geometry(kind, dims=(1.0, 1.0, 1.0)):
    """Template geometry of an analytic primitive with default ``dims``."""
    if kind not in _TEMPLATES:
        if kind == KIND_BOX:
            _TEMPLATES[kind] = box_template()
        elif kind == KIND_CYLINDER:
            _TEMPLATES[kind] = cylinder_template()
        elif kind == KIND_CAPSULE:
            _TEMPLATES[kind] = capsule_template()
        elif kind == KIND_ELLIPSOID:
            _TEMPLATES[kind] = icosphere_template(1)
        else:
            raise ValueError(kind)
    v, e = _TEMPLATES[kind]
    return Geometry(kind, np.asarray(dims, dtype=np.float32), v.copy(), e.copy(),
                    np.zeros((0, 4), dtype=np.float32))


def support(geom: Geometry, dims, u):
    """Support function max_{x in S} u . x of the exact (unsmoothed) shape.

    ``u``: (..., 3) directions in the shape's local frame.  Used only to place
    bodies at a chosen projected overlap; it is not part of the method.
    """
    u = np.asarray(u, dtype=np.float64)
    d = np.asarray(dims, dtype=np.float64)
    if geom.kind == KIND_BOX:
        return np.abs(u) @ d
    if geom.kind in (KIND_HULL, KIND_SQ_UNION):
        return (u @ geom.verts[:, :3].astype(np.float64).T).max(-1)
    if geom.kind == KIND_CAPSULE:
        return d[1] * np.abs(u[..., 2]) + d[0] * np.linalg.norm(u, axis=-1)
    if geom.kind == KIND_CYLINDER:
        return d[1] * np.abs(u[..., 2]) + d[0] * np.hypot(u[..., 0], u[..., 1])
    if geom.kind == KIND_ELLIPSOID:
        return np.linalg.norm(u * d, axis=-1)
    raise ValueError(geom.kind)


def support_point(geom: Geometry, dims, u):
    """A point of the exact (unsmoothed) shape that attains its support function in
    direction ``u`` (local frame, (3,)): argmax_{x in S} u . x (the smallest vertex index
    on ties for meshes; the +1 side of a zero component for the box and the caps).
    Used only to place bodies in contact; it is not part of the method."""
    u = np.asarray(u, dtype=np.float64)
    d = np.asarray(dims, dtype=np.float64)
    sgn = np.where(u >= 0.0, 1.0, -1.0)
    if geom.kind == KIND_BOX:
        return sgn * d
    if geom.kind in (KIND_HULL, KIND_SQ_UNION):
        v = geom.verts[:, :3].astype(np.float64)
        return v[int(np.argmax(v @ u))]
    if geom.kind == KIND_CAPSULE:
        return d[0] * u / np.linalg.norm(u) + np.array([0.0, 0.0, d[1] * sgn[2]])
    if geom.kind == KIND_CYLINDER:
        r = np.hypot(u[0], u[1])
        radial = d[0] * np.array([u[0], u[1], 0.0]) / r if r > 0 else np.zeros(3)
        return radial + np.array([0.0, 0.0, d[1] * sgn[2]])
    if geom.kind == KIND_ELLIPSOID:
        return d * d * u / np.linalg.norm(d * u)
    raise ValueError(geom.kind)


def interior_point(geom: Geometry, dims, near=None):
    """A point strictly inside the exact shape: the centre of a primitive, the vertex
    mean of a hull (inside, since the vertices are in general position).  For a union of
    superquadrics: the centre of the superquadric on whose surface ``near`` lies (the
    one whose inside-outside function is closest to 1 there); every superquadric with
    exponents <= 2 is convex, so the segment from ``near`` to that centre stays in the
    body."""
    if geom.kind == KIND_HULL:
        return geom.verts[:, :3].astype(np.float64).mean(0)
    if geom.kind == KIND_SQ_UNION:
        best, centre = np.inf, None
        for l in range(geom.n_planes // 3):
            q, t = geom.planes[3 * l].astype(np.float64), geom.planes[3 * l + 1, :3].astype(np.float64)
            e1, sc, e2 = float(geom.planes[3 * l + 1, 3]), geom.planes[3 * l + 2, :3].astype(np.float64), \
                float(geom.planes[3 * l + 2, 3])
            x = _quat_matrix(q).T @ (np.asarray(near, np.float64) - t) / sc
            f = (np.abs(x[0]) ** (2 / e2) + np.abs(x[1]) ** (2 / e2)) ** (e2 / e1) + np.abs(x[2]) ** (2 / e1)
            if abs(f - 1.0) < best:
                best, centre = abs(f - 1.0), t
        return centre
    return np.zeros(3)


def superellipsoid_surface(rings, segs, scale, eps1, eps2):
    """Mesh of one superquadric's surface in its own frame: ``rings`` latitude rings of
    ``segs`` points from the standard superellipsoid parametrisation
    (x, y, z) = (a C(eta)^eps1 C(w)^eps2, b C(eta)^eps1 S(w)^eps2, c S(eta)^eps1) with
    C(t)^e = sign(cos t)|cos t|^e and S(t)^e = sign(sin t)|sin t|^e, at
    eta_i = -pi/2 + pi (i + 1/2) / rings and w_j = 2 pi (j + 1/2) / segs (``rings`` even,
    ``segs`` a multiple of 4, so that no eta_i is 0 and no w_j a multiple of pi/2).
    Every vertex lies on the surface and none on a principal plane (x = 0, y = 0 or z = 0)
    or at a pole, where a superquadric's curvature is singular for exponents above 1 (its
    Hessian has |x~|^(2/eps - 2) terms); the polar caps are closed by their rings.  Returns (points (V, 3) float64, edges (E, 2)): ring and
    meridian edges."""
    def pw(c, e):
        return np.sign(c) * np.abs(c) ** e
    if rings % 2 or segs % 4:
        raise ValueError("rings must be even and segs a multiple of 4 (no vertex on a principal plane)")
    a, b, c = scale
    eta = -np.pi / 2 + np.pi * (np.arange(rings) + 0.5) / rings
    om = 2 * np.pi * (np.arange(segs) + 0.5) / segs
    E, W = np.meshgrid(eta, om, indexing="ij")
    pts = np.stack([a * pw(np.cos(E), eps1) * pw(np.cos(W), eps2),
                    b * pw(np.cos(E), eps1) * pw(np.sin(W), eps2),
                    c * pw(np.sin(E), eps1) * np.ones_like(W)], -1).reshape(-1, 3)
    edges = []
    for i in range(rings):
        for j in range(segs):
            edges.append((i * segs + j, i * segs + (j + 1) % segs))
            if i + 1 < rings:
                edges.append((i * segs + j, (i + 1) * segs + j))
    return pts, np.array(edges, dtype=np.int32)


def _quat_matrix(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def sq_union_geometry(prims, rings=2, segs=6):
    """A body made of superquadrics: ``prims`` is a list of (q (4,), t (3,), scale (3,),
    eps1, eps2).  The mesh is the union of the primitives' surface meshes with every
    vertex removed that lies inside the convex hull of another primitive's mesh (and the
    edges at such vertices), so that the remaining vertices sit on the body's surface."""
    from scipy.spatial import Delaunay
    pts, edges, owner = [], [], []
    for i, (q, t, sc, e1, e2) in enumerate(prims):
        p, e = superellipsoid_surface(rings, segs, sc, e1, e2)
        p = p @ _quat_matrix(q).T + np.asarray(t, np.float64)
        edges.append(e + sum(len(x) for x in pts))
        pts.append(p)
        owner.append(np.full(len(p), i))
    P, Ed, own = np.concatenate(pts), np.concatenate(edges), np.concatenate(owner)
    keep = np.ones(len(P), bool)
    for i in range(len(prims)):
        tri = Delaunay(pts[i])
        inside = tri.find_simplex(P) >= 0
        keep &= ~(inside & (own != i))
    remap = -np.ones(len(P), np.int64)
    remap[keep] = np.arange(keep.sum())
    Ed = remap[Ed]
    Ed = Ed[(Ed >= 0).all(1)].astype(np.int32)
    verts = np.zeros((int(keep.sum()), 4), np.float32)
    verts[:, :3] = P[keep]
    planes = np.zeros((3 * len(prims), 4), np.float32)
    for i, (q, t, sc, e1, e2) in enumerate(prims):
        planes[3 * i] = np.asarray(q, np.float64) / np.linalg.norm(q)
        planes[3 * i + 1] = [t[0], t[1], t[2], e1]
        planes[3 * i + 2] = [sc[0], sc[1], sc[2], e2]
    return Geometry(KIND_SQ_UNION, np.ones(3, dtype=np.float32), verts, Ed, planes)
