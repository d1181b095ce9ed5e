"""Seeded workload generators with the shapes of the paper's benchmark settings.

Every workload is a batch of independent body pairs (A, B).  Pair ``i`` names
two geometries, carries both rigid poses as ``(qw, qx, qy, qz, tx, ty, tz)``
per body, the per-body primitive dimensions and the smoothing ``tau``.

Placement (bodies always in contact): A's orientation and B's are uniform
random (Shoemake), ``t_A`` is uniform in ``[-1, 1]^3`` and a random unit
direction ``u`` is drawn.  On the exact (unsmoothed) shapes, p_A is A's support
point in direction u and c_A a point inside A; B is translated so that its
support point in direction -u lands on q = p_A + delta' w, w the unit vector
from p_A to c_A and delta' = min(delta, |c_A - p_A| / 2).  q lies in A (A is
convex and holds p_A and c_A) and in B, so the bodies intersect; moving B back
by delta' w puts its support point on p_A, where the plane u . x = u . p_A
separates the two, so the penetration depth is in (0, delta'], delta' <= delta.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .geometry import (KIND_BOX, KIND_CAPSULE, KIND_CYLINDER, KIND_ELLIPSOID,
                       Geometry, hull_from_points, interior_point, primitive_geometry, sq_union_geometry,
                       support_point)

SEED_BASE = 20261203
PRIMITIVE_KINDS = (KIND_BOX, KIND_CAPSULE, KIND_CYLINDER, KIND_ELLIPSOID)


@dataclasses.dataclass
class Workload:
    name: str
    geoms: list                 # list[Geometry]
    pair_geoms: np.ndarray      # (n, 2) int32
    poses: np.ndarray           # (n, 14) float32
    dims: np.ndarray            # (n, 6) float32
    tau: np.ndarray             # (n,) float32
    K: int = 8
    contact: np.ndarray = None  # (n, 3) float64 world point inside A and on B's surface (placement)

    @property
    def n_pairs(self):
        return int(self.pair_geoms.shape[0])

    def subset(self, idx):
        idx = np.asarray(idx)
        return Workload(self.name + "[sub]", self.geoms, self.pair_geoms[idx].copy(),
                        self.poses[idx].copy(), self.dims[idx].copy(), self.tau[idx].copy(), self.K,
                        None if self.contact is None else self.contact[idx].copy())

    def pair_counts(self):
        """(V_A, V_B, E_A, E_B) per pair."""
        nv = np.array([g.n_verts for g in self.geoms])
        ne = np.array([g.n_edges for g in self.geoms])
        a, b = self.pair_geoms[:, 0], self.pair_geoms[:, 1]
        return nv[a], nv[b], ne[a], ne[b]


def random_quaternions(rng, n):
    """Uniform random unit quaternions (Shoemake), layout (w, x, y, z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)
    return q


def _rotmat(q):
    w, x, y, z = (q / np.linalg.norm(q, axis=-1, keepdims=True)).T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _unit_vectors(rng, n):
    g = rng.normal(size=(n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _ball_points(rng, n):
    return _unit_vectors(rng, n) * rng.random(n)[:, None] ** (1.0 / 3.0)


def _place(rng, geoms, pair_geoms, dims, delta, contact_out=None):
    """Poses (n, 14) placing every pair in contact (module docstring); the common points
    q go to ``contact_out`` ((n, 3)) when given."""
    n = pair_geoms.shape[0]
    qa, qb = random_quaternions(rng, n), random_quaternions(rng, n)
    ta = rng.uniform(-1.0, 1.0, size=(n, 3))
    u = _unit_vectors(rng, n)
    Ra, Rb = _rotmat(qa), _rotmat(qb)
    tb = np.empty_like(ta)
    for i in range(n):
        ga, gb = geoms[pair_geoms[i, 0]], geoms[pair_geoms[i, 1]]
        pa = support_point(ga, dims[i, :3], Ra[i].T @ u[i])                # A's frame
        ca = interior_point(ga, dims[i, :3], near=pa)
        pb = support_point(gb, dims[i, 3:], Rb[i].T @ (-u[i]))             # B's frame
        w = Ra[i] @ (ca - pa)
        dist = np.linalg.norm(w)
        q = ta[i] + Ra[i] @ pa + min(delta[i], 0.5 * dist) * w / dist      # in A and on B
        tb[i] = q - Rb[i] @ pb
        if contact_out is not None:
            contact_out[i] = q
    poses = np.concatenate([qa, ta, qb, tb], axis=1).astype(np.float32)
    return poses


def config_box_box(n=1024, seed=SEED_BASE + 1, tau=1e-2, half=0.5):
    """Two cubes of half-extent 0.5 at ``n`` seeded relative poses."""
    rng = np.random.default_rng(seed)
    geoms = [primitive_geometry(KIND_BOX, (half, half, half))]
    pg = np.zeros((n, 2), dtype=np.int32)
    dims = np.full((n, 6), half, dtype=np.float32)
    delta = rng.uniform(0.0, 0.1, n)
    contact = np.zeros((n, 3))
    poses = _place(rng, geoms, pg, dims, delta, contact)
    return Workload("box-box", geoms, pg, poses, dims, np.full(n, tau, np.float32), contact=contact)


def _primitive_dims(rng, kind):
    d = rng.uniform(0.2, 1.0, 3)
    if kind in (KIND_CAPSULE, KIND_CYLINDER):
        d[2] = 0.0
    return d


def config_hull_vs_primitive(n=4096, seed=SEED_BASE + 2, n_points=(8, 64), log_uniform=False,
                             taus=(1e-2,), name="hull-vs-primitive"):
    """Hull of N points uniform in the unit ball (A) against a random primitive (B)."""
    rng = np.random.default_rng(seed)
    prims = {k: primitive_geometry(k) for k in PRIMITIVE_KINDS}
    geoms = [prims[k] for k in PRIMITIVE_KINDS]
    pg = np.zeros((n, 2), dtype=np.int32)
    dims = np.zeros((n, 6), dtype=np.float32)
    lo, hi = n_points
    for i in range(n):
        if log_uniform:
            m = int(np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1)))))
            m = min(max(m, lo), hi)
        else:
            m = int(rng.integers(lo, hi + 1))
        g = hull_from_points(_ball_points(rng, m))
        geoms.append(g)
        k = PRIMITIVE_KINDS[int(rng.integers(0, 4))]
        pg[i] = (len(geoms) - 1, PRIMITIVE_KINDS.index(k))
        dims[i, :3] = 1.0
        dims[i, 3:] = _primitive_dims(rng, k)
    delta = rng.uniform(0.0, 0.1, n)
    contact = np.zeros((n, 3))
    poses = _place(rng, geoms, pg, dims, delta, contact)
    tau = np.asarray(taus, dtype=np.float32)[rng.integers(0, len(taus), n)]
    return Workload(name, geoms, pg, poses, dims, tau.astype(np.float32), contact=contact)


def config_hull_vs_hull(n=64, seed=SEED_BASE + 7, n_points=(8, 64), tau=1e-2):
    """Hull against hull, each of N ~ U{8..64} points uniform in the unit ball."""
    rng = np.random.default_rng(seed)
    geoms = []
    pg = np.zeros((n, 2), dtype=np.int32)
    lo, hi = n_points
    for i in range(n):
        for side in range(2):
            geoms.append(hull_from_points(_ball_points(rng, int(rng.integers(lo, hi + 1)))))
            pg[i, side] = len(geoms) - 1
    dims = np.ones((n, 6), dtype=np.float32)
    delta = rng.uniform(0.0, 0.1, n)
    contact = np.zeros((n, 3))
    poses = _place(rng, geoms, pg, dims, delta, contact)
    return Workload("hull-vs-hull", geoms, pg, poses, dims, np.full(n, tau, np.float32), contact=contact)


def config_box_vs_sphere_hull(n=1024, seed=SEED_BASE + 3, n_sphere=32, tau=1e-2):
    """Box (dims U[0.2, 1]) against the hull of 32 points uniform on the unit sphere."""
    rng = np.random.default_rng(seed)
    geoms = [primitive_geometry(KIND_BOX)]
    pg = np.zeros((n, 2), dtype=np.int32)
    dims = np.ones((n, 6), dtype=np.float32)
    for i in range(n):
        geoms.append(hull_from_points(_unit_vectors(rng, n_sphere)))
        pg[i] = (0, len(geoms) - 1)
        dims[i, :3] = rng.uniform(0.2, 1.0, 3)
    delta = rng.uniform(0.0, 0.1, n)
    contact = np.zeros((n, 3))
    poses = _place(rng, geoms, pg, dims, delta, contact)
    return Workload("box-vs-hull32", geoms, pg, poses, dims, np.full(n, tau, np.float32), contact=contact)


def config_mixed(n=65536, seed=SEED_BASE + 4):
    """Hulls of 8..256 points (log-uniform) against mixed primitives, tau in {1e-3, 1e-2, 1e-1}."""
    return config_hull_vs_primitive(n=n, seed=seed, n_points=(8, 256), log_uniform=True,
                                    taus=(1e-3, 1e-2, 1e-1), name="mixed-uneven")


def config_mixed_pooled(n=65536, pool=4096, seed=SEED_BASE + 4):
    """The uneven mixed batch at full size with hull geometry drawn from a pool:
    ``pool`` hulls of 8..256 points (log-uniform) are built once and each of the
    ``n`` pairs picks one of them at random together with its own primitive,
    dims, tau in {1e-3, 1e-2, 1e-1} and placement (building 65536 distinct
    hulls would take minutes of qhull time on the host)."""
    rng = np.random.default_rng(seed)
    prims = {k: primitive_geometry(k) for k in PRIMITIVE_KINDS}
    geoms = [prims[k] for k in PRIMITIVE_KINDS]
    for _ in range(pool):
        m = int(np.floor(np.exp(rng.uniform(np.log(8), np.log(257)))))
        geoms.append(hull_from_points(_ball_points(rng, min(max(m, 8), 256))))
    pg = np.zeros((n, 2), dtype=np.int32)
    pg[:, 0] = 4 + rng.integers(0, pool, n)
    kinds = rng.integers(0, 4, n)
    pg[:, 1] = kinds
    dims = np.ones((n, 6), dtype=np.float32)
    d = rng.uniform(0.2, 1.0, size=(n, 3))
    d[np.isin(kinds, [1, 2]), 2] = 0.0            # capsule / cylinder use (r, h)
    dims[:, 3:] = d
    delta = rng.uniform(0.0, 0.1, n)
    contact = np.zeros((n, 3))
    poses = _place(rng, geoms, pg, dims, delta, contact)
    tau = np.asarray((1e-3, 1e-2, 1e-1), dtype=np.float32)[rng.integers(0, 3, n)]
    return Workload("mixed-uneven-pooled", geoms, pg, poses, dims, tau, contact=contact)


SQ_RESOLUTIONS = ((4, 12), (4, 8), (2, 12), (2, 8), (2, 4))


def random_sq_union(rng, n_prims, step=0.22, scale=(0.12, 0.28), eps=(0.3, 1.5), max_verts=256,
                    max_edges=768):
    """A blob of ``n_prims`` superquadrics: each centre is a step of length ``step`` from
    an earlier primitive's centre (a random tree, like limbs on a body), axis lengths and
    both exponents uniform, orientations uniform; centred on the mean of the centres.
    The mesh resolution is the finest that stays within the per-geometry limits."""
    c = np.zeros((n_prims, 3))
    for i in range(1, n_prims):
        c[i] = c[rng.integers(0, i)] + step * _unit_vectors(rng, 1)[0]
    c -= c.mean(0)
    q = random_quaternions(rng, n_prims)
    sc = rng.uniform(scale[0], scale[1], size=(n_prims, 3))
    e = rng.uniform(eps[0], eps[1], size=(n_prims, 2))
    prims = [(q[i], c[i], sc[i], float(e[i, 0]), float(e[i, 1])) for i in range(n_prims)]
    # the finest per-primitive mesh whose pruned union fits 256 vertices and 768 edges
    for rings, segs in SQ_RESOLUTIONS:
        g = sq_union_geometry(prims, rings, segs)
        if g.n_verts <= max_verts and g.n_edges <= max_edges:
            return g
    raise ValueError("too many primitives for the mesh limits")


def config_sq_union(n=1024, n_prims=18, pool=8, seed=SEED_BASE + 6, tau=1e-2):
    """Pairs of multi-superquadric bodies (the paper's armadillo setting, Sec. V, with
    synthetic primitive sets): a pool of bodies of ``n_prims`` primitives each, pairs
    drawn from it at seeded poses with projected overlap U[0, 0.1]."""
    rng = np.random.default_rng(seed)
    geoms = [random_sq_union(rng, n_prims) for _ in range(pool)]
    pg = rng.integers(0, pool, size=(n, 2)).astype(np.int32)
    dims = np.ones((n, 6), dtype=np.float32)
    delta = rng.uniform(0.0, 0.1, n)
    contact = np.zeros((n, 3))
    poses = _place(rng, geoms, pg, dims, delta, contact)
    return Workload(f"sq-union{n_prims}", geoms, pg, poses, dims, np.full(n, tau, np.float32), contact=contact)


def serving_trace(seed=SEED_BASE + 5, rate=2000.0, duration=10.0, max_pairs=8192):
    """Poisson arrivals; request sizes log-uniform in [1, max_pairs]; fwd or fwd+bwd 50/50.

    Returns a list of ``(arrival_s, n_pairs, with_backward)``.
    """
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        m = int(np.floor(np.exp(rng.uniform(0.0, np.log(max_pairs + 1)))))
        out.append((t, max(1, min(m, max_pairs)), bool(rng.integers(0, 2))))
    return out


def make_config(idx, n=None):
    """Workload of one of the benchmark settings by index (1..4), optionally resized."""
    if idx == 1:
        return config_box_box(n or 1024)
    if idx == 2:
        return config_hull_vs_primitive(n or 4096)
    if idx == 3:
        return config_box_vs_sphere_hull(n or 1024)
    if idx == 4:
        return config_mixed(n or 65536)
    raise ValueError(idx)
