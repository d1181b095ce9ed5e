"""The seeded placement puts every pair in contact, checked on the exact shapes.

The generators place body B so that its support point in direction -u lands on a
point q inside body A (at most delta = U[0, 0.1] from A's own support point, on
the segment towards A's interior), and keep q.  Here q is checked with the
textbook exact (unsmoothed) signed distances, written out independently of the
generators: q must lie inside A, no deeper than 0.1, and on B's surface (up to
the FP32 rounding of the stored poses).  These inputs stand in for the paper's
colliding pairs (the Sec. V validity experiments use touching bodies).
"""
import numpy as np
import pytest

import synth


def _rot(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def exact_sdf(geom, dims, x):
    """Exact signed distance of the unsmoothed shape at local point x (hulls: the largest
    plane value, which is the exact distance for points inside); for an ellipsoid the
    value of |x~| - 1 scaled by the smallest semi-axis (same sign as the distance,
    within a factor of the axis ratio in magnitude)."""
    d = np.asarray(dims, np.float64)
    if geom.kind == synth.KIND_BOX:
        q = np.abs(x) - d
        return np.linalg.norm(np.maximum(q, 0.0)) + min(q.max(), 0.0)
    if geom.kind == synth.KIND_HULL:
        P = geom.planes.astype(np.float64)
        return float((P[:, :3] @ x - P[:, 3]).max())
    if geom.kind == synth.KIND_CAPSULE:
        z = np.clip(x[2], -d[1], d[1])
        return np.linalg.norm(x - np.array([0.0, 0.0, z])) - d[0]
    if geom.kind == synth.KIND_CYLINDER:
        q = np.array([np.hypot(x[0], x[1]) - d[0], abs(x[2]) - d[1]])
        return np.linalg.norm(np.maximum(q, 0.0)) + min(q.max(), 0.0)
    if geom.kind == synth.KIND_ELLIPSOID:
        return (np.linalg.norm(x / d) - 1.0) * d.min()
    raise ValueError(geom.kind)


WORKLOADS = {
    "box-box": lambda: synth.config_box_box(n=256),
    "hull-vs-primitive": lambda: synth.config_hull_vs_primitive(n=256),
    "box-vs-hull32": lambda: synth.config_box_vs_sphere_hull(n=128),
    "mixed": lambda: synth.config_mixed(n=256, seed=99),
    "hull-vs-hull": lambda: synth.config_hull_vs_hull(n=64),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_every_pair_touches(name):
    w = WORKLOADS[name]()
    assert w.contact is not None and w.contact.shape == (w.n_pairs, 3)
    for i in range(w.n_pairs):
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
        P = w.poses[i].astype(np.float64)
        q = w.contact[i]
        xa = _rot(P[:4]).T @ (q - P[4:7])
        xb = _rot(P[7:11]).T @ (q - P[11:14])
        phi_a = exact_sdf(ga, w.dims[i, :3], xa)
        phi_b = exact_sdf(gb, w.dims[i, 3:], xb)
        assert -0.1 <= phi_a <= 1e-6, (i, phi_a)          # inside A, at most 0.1 deep
        assert abs(phi_b) <= 2e-6, (i, phi_b)              # on B's surface


def test_depth_spreads_over_the_range():
    """The common point's depth in A follows delta = U[0, 0.1] (scaled by how the segment
    towards A's interior meets A's faces): not all shallow, not all deep."""
    w = synth.config_box_box(n=512)
    depth = []
    for i in range(w.n_pairs):
        P = w.poses[i].astype(np.float64)
        xa = _rot(P[:4]).T @ (w.contact[i] - P[4:7])
        depth.append(-exact_sdf(w.geoms[0], w.dims[i, :3], xa))
    depth = np.array(depth)
    # box corner: the segment towards the centre runs along the diagonal, depth = delta / sqrt 3
    assert depth.max() <= 0.1 / np.sqrt(3) + 1e-6
    assert (depth > 0.03).mean() > 0.4 and (depth < 0.01).mean() > 0.1


def test_placement_is_deterministic():
    """The same seed gives the same pairs, poses and common points."""
    a = synth.config_hull_vs_primitive(n=64)
    b = synth.config_hull_vs_primitive(n=64)
    np.testing.assert_array_equal(a.pair_geoms, b.pair_geoms)
    np.testing.assert_array_equal(a.poses, b.poses)
    np.testing.assert_array_equal(a.contact, b.contact)
