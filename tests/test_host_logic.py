"""Host-side logic of the C ABI on a host-only context (no GPU needed): geometry
validation, argument errors and the refusal of device work."""
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


def add(api, ctx, g, **over):
    d = dict(kind=g.kind, dims=g.dims, verts=g.verts, edges=g.edges, planes=g.planes if len(g.planes) else None)
    d.update(over)
    return api.cm_create_geometry(ctx, d["kind"], d["dims"], d["verts"], d["edges"], d["planes"])


def test_valid_geometries_get_consecutive_ids(api, ctx):
    w = synth.make_config(2, 4)
    ids = [add(api, ctx, g) for g in w.geoms]
    assert ids == list(range(len(w.geoms)))
    assert api.cm_num_geometries(ctx) == len(w.geoms)


@pytest.mark.parametrize("case", ["kind", "edge_index", "degenerate_edge", "nan_vertex", "dims", "planes_on_box",
                                  "hull_without_planes", "non_unit_plane", "too_many_verts", "too_many_edges"])
def test_invalid_geometry_is_rejected(api, ctx, case):
    box = synth.primitive_geometry(synth.KIND_BOX, (0.5, 0.5, 0.5))
    hull = synth.hull_from_points(np.random.default_rng(0).normal(size=(20, 3)))
    over, g = {}, box
    if case == "kind":
        over = dict(kind=7)
    elif case == "edge_index":
        e = box.edges.copy()
        e[0, 1] = 8
        over = dict(edges=e)
    elif case == "degenerate_edge":
        e = box.edges.copy()
        e[0, 1] = e[0, 0]
        over = dict(edges=e)
    elif case == "nan_vertex":
        v = box.verts.copy()
        v[3, 1] = np.nan
        over = dict(verts=v)
    elif case == "dims":
        over = dict(dims=(0.5, -1.0, 0.5))
    elif case == "planes_on_box":
        over = dict(planes=hull.planes)
    elif case == "hull_without_planes":
        g, over = hull, dict(planes=None)
    elif case == "non_unit_plane":
        p = hull.planes.copy()
        p[0, :3] *= 2
        g, over = hull, dict(planes=p)
    elif case == "too_many_verts":
        g, over = hull, dict(verts=np.zeros((257, 4), np.float32))
    elif case == "too_many_edges":
        g, over = hull, dict(edges=np.zeros((769, 2), np.int32) + np.array([0, 1], np.int32))
    with pytest.raises(api.CMError) as ei:
        add(api, ctx, g, **over)
    assert ei.value.status == api.CM_ERR_INVALID_ARG and api.cm_last_error()
    assert api.cm_num_geometries(ctx) == 0


def test_host_only_context_refuses_device_work(api, ctx):
    add(api, ctx, synth.primitive_geometry(synth.KIND_BOX, (0.5, 0.5, 0.5)))
    with pytest.raises(api.CMError) as ei:
        api.cm_sync_geometry(ctx)
    assert ei.value.status == api.CM_ERR_INVALID_ARG and "host-only" in str(ei.value)
    with pytest.raises(api.CMError):
        api.cm_server_start(ctx, api.cm_default_params(), 1024, 2)
    api.cm_check_device_error(ctx)                  # nothing ran, nothing to report


def test_bad_params_are_rejected_before_any_work(api, ctx):
    import ctypes
    lib = api._lib
    add(api, ctx, synth.primitive_geometry(synth.KIND_BOX, (0.5, 0.5, 0.5)))
    for over in (dict(tau=0.0), dict(tau=float("nan")), dict(w_reg=0.0), dict(K=0), dict(K=17), dict(flags=8),
                 dict(eps_min=-1.0)):
        p = api.cm_default_params(**over)
        st = lib.cm_contact_manifold_fwd(ctx, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None, None,
                                         ctypes.byref(p), ctypes.c_void_p(8), None)
        assert st == api.CM_ERR_INVALID_ARG, over
    p = api.cm_default_params()
    assert lib.cm_contact_manifold_fwd(ctx, -1, None, None, None, None, ctypes.byref(p), None, None) == \
        api.CM_ERR_INVALID_ARG
    assert lib.cm_contact_manifold_fwd(ctx, 0, None, None, None, None, ctypes.byref(p), None, None) == api.CM_OK
    assert lib.cm_contact_manifold_fwd(ctx, 3, None, None, None, None, ctypes.byref(p), None, None) == \
        api.CM_ERR_INVALID_ARG


def sq_body(seed=0, n=4):
    return synth.random_sq_union(np.random.default_rng(seed), n)


def test_sq_union_geometry_is_accepted(api, ctx):
    ids = [add(api, ctx, sq_body(s, n)) for s, n in ((0, 1), (1, 5), (2, 18))]
    assert ids == [0, 1, 2]


@pytest.mark.parametrize("case", ["rows", "eps_high", "eps_low", "zero_quat", "scale", "too_many", "nan"])
def test_invalid_sq_union_is_rejected(api, ctx, case):
    g = sq_body()
    P = g.planes.copy()
    if case == "rows":
        P = P[:-1]
    elif case == "eps_high":
        P[1, 3] = 2.5
    elif case == "eps_low":
        P[5, 3] = 0.05
    elif case == "zero_quat":
        P[0] = 0.0
    elif case == "scale":
        P[2, 1] = -0.2
    elif case == "too_many":
        P = np.concatenate([P] * 9)           # 36 superquadrics
    elif case == "nan":
        P[4, 0] = np.nan
    with pytest.raises(api.CMError) as ei:
        add(api, ctx, g, planes=P)
    assert ei.value.status == api.CM_ERR_INVALID_ARG and api.cm_last_error()
    assert api.cm_num_geometries(ctx) == 0


def test_selection_and_tracing_limits(api, ctx):
    import ctypes
    lib = api._lib
    add(api, ctx, synth.primitive_geometry(synth.KIND_BOX, (0.5, 0.5, 0.5)))
    for over in (dict(top_edges=33), dict(top_verts=-1), dict(trace_iters=9), dict(trace_iters=-1)):
        p = api.cm_default_params(**over)
        st = lib.cm_contact_manifold_fwd(ctx, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None, None,
                                         ctypes.byref(p), ctypes.c_void_p(8), None)
        assert st == api.CM_ERR_INVALID_ARG, over
    assert api.cm_default_params().trace_iters == 0


def test_destroy_geometry(api, ctx):
    """Unregistering keeps ids stable (never reused), rejects unknown and twice-destroyed
    ids, and new geometry still gets the next id."""
    w = synth.make_config(2, 4)
    ids = [add(api, ctx, g) for g in w.geoms]
    api.cm_destroy_geometry(ctx, ids[1])
    assert api.cm_num_geometries(ctx) == len(ids)
    for bad in (ids[1], -1, len(ids)):
        with pytest.raises(api.CMError) as ei:
            api.cm_destroy_geometry(ctx, bad)
        assert ei.value.status == api.CM_ERR_INVALID_ARG
    assert add(api, ctx, w.geoms[0]) == len(ids)


def test_bench_oracle_rate_restores_thread_count():
    """The benchmark's CPU-baseline leg times the oracle on one thread and on the default
    intra-op pool; the single-thread leg leaves the pool as it found it."""
    import torch
    import bench
    import synth
    w = synth.make_config(1, 4)
    before = torch.get_num_threads()
    r, n, dt, cores = bench.cpu_oracle_rate(w, budget_s=30.0, max_pairs=2, threads=1)
    assert cores == 1 and n == 2 and r > 0
    assert torch.get_num_threads() == before


def test_bench_alu_roofline_object():
    """The benchmark's roofline object: both pipes against the peaks from unit counts and
    the 2070 MHz clock, the larger fraction binding, the measured loop throughputs beside;
    the adjoint's work is the forward's plus the reverse's."""
    import bench
    import synth
    w = synth.make_config(2, 16)
    assert abs(bench.FP32_PEAK_DERIVED - 152 * 128 * 2 * 2.07e9) < 1.0
    assert abs(bench.MUFU_PEAK_DERIVED - 152 * 32 * 2.07e9) < 1.0
    assert bench.alu_peaks(76)[0] == bench.FP32_PEAK_DERIVED / 2
    for backward in (False, True):
        r = bench.alu_roofline(w, 1e-5, (76e12, 9.8e12), backward=backward)
        assert r["bound"] == "alu" and r["pipe"] in ("fp32", "mufu")
        for k, p in r["pipes"].items():
            scale = 1e12 if k == "fp32" else 1e9
            assert abs(p["frac"] - p["achieved"] / p["peak"]) < 1e-12
            assert abs(p["frac_of_measured"] - p["achieved"] * scale / (76e12 if k == "fp32" else 9.8e12)) < 1e-12
        assert r["frac"] == max(p["frac"] for p in r["pipes"].values())
        assert r["traffic"] is None
    assert bench.alu_roofline(w, 1e-5, (1, 1))["algorithmic_bytes"] == 348 * 16
    fl_b, mu_b = bench.bwd_work_per_pair(w)
    fl_f, mu_f = bench.fp32_flops_per_pair(w), bench.mufu_ops_per_pair(w)
    # the reverse adds work on both pipes; a hull's reverse needs no transcendental per
    # plane (its moments come from the forward pass), so the adjoint's MUFU work grows
    # less than its FP32 work
    assert (fl_b > 1.5 * fl_f).all() and (mu_b > 1.1 * mu_f).all()
    assert ((mu_b / mu_f) < (fl_b / fl_f)).all()


def test_bench_cpu_baseline_leg():
    """The benchmark's cpu_baseline object: the over-pairs value with the intra-op and
    single-thread figures beside it, every figure positive, forward and backward."""
    import bench
    import synth
    w = synth.make_config(1, 8)
    cpu = bench.cpu_baseline_leg(w, cpu_seconds=1.0, pool_budget_s=1.0)
    assert cpu["kind"] == "oracle" and cpu["unit"] == "pairs/s" and "over_pairs_error" not in cpu
    assert cpu["value"] > 0 and cpu["cores"] >= 1 and "single-threaded processes" in cpu["sample"]
    assert "forward + backward" in cpu["sample"]
    for k in ("intra_op_threads", "single_thread"):
        assert cpu[k]["value"] > 0 and cpu[k]["unit"] == "pairs/s"


def test_bench_oracle_over_pairs_pool():
    """The pair-parallel oracle timing: single-threaded spawned processes, each on its own
    share of the pairs, returning a positive rate within its time limit."""
    import bench
    import synth
    w = synth.make_config(1, 16)
    r, pairs, span, procs = bench.cpu_oracle_rate_over_pairs(w, budget_s=1.0, procs=2, timeout_s=120.0)
    assert procs == 2 and 0 < pairs <= 16 and span > 0 and r > 0


def test_bench_headline_sample_is_seeded():
    """The oracle's 1 % sample of the headline batch: seeded, the same pairs every time."""
    import bench
    import synth
    w = synth.config_hull_vs_primitive(n=300, seed=5)
    a, b = bench.oracle_sample(w), bench.oracle_sample(w)
    assert a.n_pairs == 3
    np.testing.assert_array_equal(a.poses, b.poses)
