"""The library's own convex hull (cm_create_hull_geometry) and the geometry read-back
(cm_get_geometry), on a host-only context: no GPU needed.  The hull is compared with
qhull's (scipy), the input generator's hull, on point sets in general position, and
checked on a cube (coplanar facets, repeated points) and on degenerate inputs."""
import numpy as np
import pytest

import synth


@pytest.fixture()
def api():
    from paper_2602_20304_gb300 import build_lib
    build_lib.build()
    from paper_2602_20304_gb300 import api
    return api


@pytest.fixture()
def ctx(api):
    c = api.cm_create_context(-1)
    yield c
    api.cm_destroy_context(c)


def ball_points(seed, n):
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return u * rng.uniform(0, 1, (n, 1)) ** (1 / 3)


def match_planes(a, b, tol=1e-6):
    """Every plane of ``a`` equals one plane of ``b`` and vice versa (same count)."""
    assert a.shape == b.shape
    used = np.zeros(len(b), dtype=bool)
    for p in a:
        d = np.abs(b - p).max(1)
        d[used] = np.inf
        j = int(np.argmin(d))
        assert d[j] <= tol, (p, b[j])
        used[j] = True


@pytest.mark.parametrize("n,seed", [(8, 0), (20, 1), (64, 2), (200, 3), (5000, 4)])
def test_hull_equals_qhull_in_general_position(api, ctx, n, seed):
    pts = ball_points(seed, n)
    if n > 1000:   # many interior points around a hull that fits the vertex limit
        pts = np.concatenate([0.5 * pts, ball_points(seed + 100, 150)])
        pts = pts[np.random.default_rng(seed).permutation(len(pts))]
    gid = api.cm_create_hull_geometry(ctx, pts)
    got = api.cm_get_geometry(ctx, gid)
    ref = synth.hull_from_points(pts)
    assert got["kind"] == api.CM_HULL
    np.testing.assert_array_equal(got["verts"], ref.verts)
    np.testing.assert_array_equal(got["edges"], ref.edges)
    match_planes(got["planes"], ref.planes)


def test_hull_is_closed_convex_and_contains_its_points(api, ctx):
    pts = ball_points(9, 300)
    g = api.cm_get_geometry(ctx, api.cm_create_hull_geometry(ctx, pts))
    V, E, F = len(g["verts"]), len(g["edges"]), len(g["planes"])
    assert V - E + F == 2 and 2 * E == 3 * F            # closed sphere of triangles (no flat facets here)
    n, o = g["planes"][:, :3].astype(np.float64), g["planes"][:, 3].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)
    assert (pts @ n.T - o).max() <= 1e-6                # every input point inside every plane
    on = np.abs(g["verts"][:, :3].astype(np.float64) @ n.T - o) <= 1e-6
    assert (on.sum(0) == 3).all()                       # each plane through its triangle's three vertices


def test_cube_with_repeated_and_interior_points(api, ctx):
    """A cube's corners (each face built from two coplanar triangles, merged into one
    facet), repeated corners and interior points: the 8 corners in first-occurrence
    order, the 12 cube edges (no face diagonals) and 6 planes, one per face, with normals
    +-e_i and offset 1."""
    rng = np.random.default_rng(5)
    corners = np.array([[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)])
    inner = rng.uniform(-0.9, 0.9, (20, 3))
    pts = np.concatenate([inner[:10], corners[::-1], inner[10:], corners])
    g = api.cm_get_geometry(ctx, api.cm_create_hull_geometry(ctx, pts))
    np.testing.assert_array_equal(g["verts"][:, :3], corners[::-1])
    assert len(g["edges"]) == 12 and len(g["planes"]) == 6
    n, o = g["planes"][:, :3], g["planes"][:, 3]
    np.testing.assert_allclose(o, 1.0, atol=1e-7)
    axes = np.concatenate([np.eye(3), -np.eye(3)])
    for a in axes:
        assert int((np.abs(n - a).max(1) < 1e-7).sum()) == 1
    lengths = np.linalg.norm(np.diff(g["verts"][g["edges"]][:, :, :3], axis=1)[:, 0], axis=1)
    np.testing.assert_allclose(lengths, 2.0, atol=1e-6)
    ref = synth.hull_from_points(pts)                  # the generator merges the same way
    np.testing.assert_array_equal(g["verts"], ref.verts)
    np.testing.assert_array_equal(g["edges"], ref.edges)
    match_planes(g["planes"], ref.planes)


@pytest.mark.parametrize("case", ["three", "equal", "collinear", "coplanar", "nan", "too_many"])
def test_degenerate_point_sets_are_rejected(api, ctx, case):
    rng = np.random.default_rng(6)
    pts = {
        "three": rng.normal(size=(3, 3)),
        "equal": np.ones((10, 3)),
        "collinear": np.outer(rng.normal(size=12), [1.0, 2.0, 3.0]),
        "coplanar": np.concatenate([rng.normal(size=(12, 2)), np.zeros((12, 1))], 1),
        "nan": np.concatenate([rng.normal(size=(9, 3)), [[np.nan, 0, 0]]]),
        "too_many": (lambda u: u / np.linalg.norm(u, axis=1, keepdims=True))(rng.normal(size=(300, 3))),
    }[case]
    with pytest.raises(api.CMError) as ei:
        api.cm_create_hull_geometry(ctx, pts)
    assert ei.value.status == api.CM_ERR_INVALID_ARG
    assert api.cm_num_geometries(ctx) == 0


def test_get_geometry_returns_what_was_registered(api, ctx):
    w = synth.make_config(2, 3)
    for g in w.geoms:
        gid = api.cm_create_geometry(ctx, g.kind, g.dims, g.verts, g.edges,
                                     g.planes if len(g.planes) else None)
        got = api.cm_get_geometry(ctx, gid)
        assert got["kind"] == g.kind
        np.testing.assert_array_equal(got["dims"], g.dims)
        np.testing.assert_array_equal(got["verts"], g.verts)
        np.testing.assert_array_equal(got["edges"], g.edges)
        np.testing.assert_array_equal(got["planes"], g.planes if g.kind == synth.KIND_HULL else np.zeros((0, 4)))
    api.cm_destroy_geometry(ctx, 0)
    for bad in (0, -1, api.cm_num_geometries(ctx)):
        with pytest.raises(api.CMError) as ei:
            api.cm_get_geometry(ctx, bad)
        assert ei.value.status == api.CM_ERR_INVALID_ARG


def same_mesh_up_to_order(got, ref_verts, ref_edges, tol=1e-6):
    """The two meshes have the same vertex rows (matched one to one within ``tol``) and,
    through that matching, the same edge set."""
    gv, rv = got["verts"].astype(np.float64), np.asarray(ref_verts, dtype=np.float64)
    assert gv.shape == rv.shape
    to_ref = np.full(len(gv), -1)
    for i, row in enumerate(gv):
        d = np.abs(rv - row).max(1)
        j = int(np.argmin(d))
        assert d[j] <= tol, (i, row, rv[j])
        to_ref[i] = j
    assert len(set(to_ref.tolist())) == len(gv)
    ge = {tuple(sorted((int(to_ref[a]), int(to_ref[b])))) for a, b in got["edges"]}
    re_ = {tuple(sorted((int(a), int(b)))) for a, b in np.asarray(ref_edges)}
    assert len(ge) == len(got["edges"]) and ge == re_


@pytest.mark.parametrize("kind,tess,nv,ne", [
    (synth.KIND_BOX, 0, 8, 12),
    (synth.KIND_CYLINDER, 16, 32, 48), (synth.KIND_CYLINDER, 7, 14, 21),
    (synth.KIND_CAPSULE, 16, 66, 144), (synth.KIND_CAPSULE, 5, 22, 45),
    (synth.KIND_ELLIPSOID, 0, 12, 30), (synth.KIND_ELLIPSOID, 1, 42, 120), (synth.KIND_ELLIPSOID, 2, 162, 480)])
def test_primitive_meshes_equal_the_generator_templates(api, ctx, kind, tess, nv, ne):
    """The library's primitive meshes are the input generator's templates (the same unit
    rows and edges, vertex order aside) at the resolutions the settings use and others."""
    dims = (0.5, 0.3, 0.2)
    g = api.cm_get_geometry(ctx, api.cm_create_primitive_geometry(ctx, kind, dims, tess))
    assert g["kind"] == kind and len(g["verts"]) == nv and len(g["edges"]) == ne
    np.testing.assert_array_equal(g["dims"], np.float32(dims))
    ref = {synth.KIND_BOX: lambda: synth.box_template(),
           synth.KIND_CYLINDER: lambda: synth.cylinder_template(tess),
           synth.KIND_CAPSULE: lambda: synth.capsule_template(tess),
           synth.KIND_ELLIPSOID: lambda: synth.icosphere_template(tess)}[kind]()
    same_mesh_up_to_order(g, *ref)
    # the unit rows lie on the unit template surface
    u = g["verts"][:, :3].astype(np.float64)
    if kind == synth.KIND_ELLIPSOID:
        np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-6)
    if kind == synth.KIND_CYLINDER:
        np.testing.assert_allclose(np.hypot(u[:, 0], u[:, 1]), 1.0, atol=1e-6)
    if kind == synth.KIND_CAPSULE:
        np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-6)
        assert (np.sign(g["verts"][:, 3]) * u[:, 2] >= -1e-7).all()   # each cap's rows on its side


@pytest.mark.parametrize("kind,tess,dims", [
    (synth.KIND_CYLINDER, 2, (1, 1, 0)), (synth.KIND_CYLINDER, 129, (1, 1, 0)),
    (synth.KIND_CAPSULE, 64, (1, 1, 0)), (synth.KIND_ELLIPSOID, 3, (1, 1, 1)),
    (synth.KIND_HULL, 0, (1, 1, 1)), (synth.KIND_BOX, 0, (1, -1, 1)), (7, 0, (1, 1, 1))])
def test_primitive_arguments_are_checked(api, ctx, kind, tess, dims):
    with pytest.raises(api.CMError) as ei:
        api.cm_create_primitive_geometry(ctx, kind, dims, tess)
    assert ei.value.status == api.CM_ERR_INVALID_ARG
    assert api.cm_num_geometries(ctx) == 0


def test_coplanar_rims_give_a_closed_hull_of_flat_facets(api, ctx):
    """Two rims of 16 points (every cap 16 coplanar points): all 32 are vertices, each cap
    is one facet (normal -+z) and the side 16 rectangles, 48 edges (the rims and the 16
    vertical edges, no diagonals)."""
    t = 2 * np.pi * np.arange(16) / 16
    pts = np.concatenate([np.stack([np.cos(t), np.sin(t), np.full(16, z)], 1) for z in (-0.5, 0.5)])
    g = api.cm_get_geometry(ctx, api.cm_create_hull_geometry(ctx, pts))
    V, E, F = len(g["verts"]), len(g["edges"]), len(g["planes"])
    assert (V, E, F) == (32, 48, 18)
    n = g["planes"][:, :3]
    assert int((np.abs(n[:, 2] - 1) < 1e-6).sum()) == 1 and int((np.abs(n[:, 2] + 1) < 1e-6).sum()) == 1
    assert int((np.abs(n[:, 2]) < 1e-6).sum()) == 16
    assert (pts @ n.T.astype(np.float64) - g["planes"][:, 3]).max() <= 1e-6


@pytest.mark.parametrize("seed", range(12))
def test_nearly_degenerate_sets_give_a_closed_hull_or_a_clean_refusal(api, ctx, seed):
    """Cube corners jittered by 1e-12, repeated, with points on the faces and inside:
    either the cube (8 vertices, 12 edges, 6 facets) containing every point, or
    CM_ERR_INVALID_ARG."""
    rng = np.random.default_rng(seed)
    corners = np.array([[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)])
    face = rng.uniform(-1, 1, (30, 3))
    face[np.arange(30), rng.integers(0, 3, 30)] = rng.choice([-1.0, 1.0], 30)
    pts = np.concatenate([corners, corners + 1e-12 * rng.normal(size=(8, 3)), face, rng.uniform(-1, 1, (30, 3))])
    pts = pts[rng.permutation(len(pts))]
    try:
        g = api.cm_get_geometry(ctx, api.cm_create_hull_geometry(ctx, pts))
    except api.CMError as e:
        assert e.status == api.CM_ERR_INVALID_ARG
        return
    V, E, F = len(g["verts"]), len(g["edges"]), len(g["planes"])
    assert (V, E, F) == (8, 12, 6)
    n, o = g["planes"][:, :3].astype(np.float64), g["planes"][:, 3].astype(np.float64)
    assert (pts @ n.T - o).max() <= 1e-6


def test_cube_corner_hull_manifold_equals_the_box_primitive():
    """The hull of the 8 corners of [-0.5, 0.5]^3 has the box's 6 planes and 12 edges, so its
    smooth SDF (LSE over planes, Sec. IV-B2) is the BOX primitive's and the oracle gives the
    same manifold for it as for a BOX of half-extent 0.5 (a face split into two equal planes
    would shift the SDF by tau ln 2 = 6.9e-3 at tau = 1e-2)."""
    import oracle
    corners = 0.5 * np.array([[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)])
    hull = synth.hull_from_points(corners)
    assert (hull.n_verts, hull.n_edges, hull.n_planes) == (8, 12, 6)
    w = synth.config_hull_vs_primitive(n=12, seed=31)
    box = synth.primitive_geometry(synth.KIND_BOX)
    # A = the box (as a primitive of half-extent 0.5, then as the cube-corner hull), B as drawn
    geoms = [box, hull] + w.geoms
    pg_box = np.stack([np.zeros(w.n_pairs, np.int32), 2 + w.pair_geoms[:, 1]], 1)
    pg_hull = np.stack([np.ones(w.n_pairs, np.int32), 2 + w.pair_geoms[:, 1]], 1)
    dims = w.dims.copy()
    dims[:, :3] = 0.5
    a = oracle.batch_manifold(geoms, pg_box, w.poses, dims, w.tau)
    b = oracle.batch_manifold(geoms, pg_hull, w.poses, dims, w.tau)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-9)
