"""Candidate-level parity: every vertex-SDF candidate (Sec. IV-C) and every edge-pair
witness candidate (Sec. IV-D3) the kernel reduces a manifold from, dumped through the C ABI
and compared row by row with the FP64 oracle's candidates.  Each field of each candidate is
held to the fixed tolerance (1e-5 on p and d, 1e-4 on n and w) or, where it misses it, to
16 times the largest move of the oracle's own candidate when every FP32 input of the pair
moves by one ulp (four draws; the per-pair bar of the manifold tests, per candidate)."""
import numpy as np
import pytest
import torch

import synth
from _parity import BOUND_FACTOR, SLICES, TOL, ULP_DRAWS, nudged, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    from paper_2602_20304_gb300.engine import Engine
    e = Engine(0)
    yield e
    e.close()


def oracle_candidates(w, params, i):
    from oracle.manifold import pair_candidates
    from oracle.preselect import pair_candidates_preselect
    t = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa: E731
    ga, gb = w.geoms[int(w.pair_geoms[i, 0])], w.geoms[int(w.pair_geoms[i, 1])]
    with torch.no_grad():
        if params.top_verts or params.top_edges:
            c = pair_candidates_preselect(ga, gb, t(w.poses[i]), t(w.dims[i]), float(w.tau[i]), oracle_params(params),
                                          params.top_verts, params.top_edges)
        else:
            c = pair_candidates(ga, gb, t(w.poses[i]), t(w.dims[i]), float(w.tau[i]), oracle_params(params))
    return c.numpy()


def to_oracle_order(rows, nvs):
    """Kernel ids (vertices, then both witnesses of each edge pair interleaved) -> the
    oracle's order (vertices, first witnesses of every edge pair, then second ones)."""
    return np.concatenate([rows[:nvs], rows[nvs::2], rows[nvs + 1::2]])


def check_candidates(engine, w, params, idx, what):
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    out, cand, off = engine.forward_dump(pg, poses, dims, tau, params)
    plain = engine.forward(pg, poses, dims, tau, params)
    torch.cuda.synchronize()
    engine.check()
    assert torch.allclose(out, plain, atol=1e-6, rtol=0), "the dump changed the manifold"
    cand = cand.cpu().numpy().astype(np.float64)
    n_rows, n_within, worst = 0, 0, 0.0
    for i in idx:
        ref = oracle_candidates(w, params, i)
        rows = cand[off[i]:off[i + 1]]
        assert rows.shape == ref.shape, (i, rows.shape, ref.shape)
        nvs = len(rows) - 2 * _n_edge_pairs(w, params, i)
        got = to_oracle_order(rows, nvs) if nvs < len(rows) else rows
        err = {f: np.abs(got[:, s] - ref[:, s]).max(1) for f, s in SLICES.items()}
        miss = np.zeros(len(ref), bool)
        for f in SLICES:
            miss |= err[f] > TOL[f]
        n_rows += len(ref)
        n_within += int((~miss).sum())
        if miss.any():
            spread = {f: np.zeros(int(miss.sum())) for f in SLICES}
            rng = np.random.default_rng(int(i))
            for _ in range(ULP_DRAWS):
                wn = nudged(w, [i], rng)
                refn = oracle_candidates(wn, params, 0)[miss]
                for f, s in SLICES.items():
                    spread[f] = np.maximum(spread[f], np.abs(refn[:, s] - ref[miss][:, s]).max(1))
            for f in SLICES:
                bound = np.maximum(TOL[f], BOUND_FACTOR * spread[f])
                assert (err[f][miss] <= bound).all(), (what, int(i), f, float((err[f][miss] / bound).max()))
                worst = max(worst, float((err[f][miss] / bound).max()))
    info = {"pairs": len(idx), "candidates": n_rows, "within_tol": n_within / n_rows, "worst_over_bound": worst}
    print(what, info)
    assert n_within / n_rows >= 0.95          # a sanity floor; the per-candidate bound above is the bar
    return info


def _n_edge_pairs(w, params, i):
    if params.flags & 3:
        return 0
    ga, gb = w.geoms[int(w.pair_geoms[i, 0])], w.geoms[int(w.pair_geoms[i, 1])]
    ea, eb = ga.n_edges, gb.n_edges
    if params.top_edges:
        ea, eb = min(params.top_edges, ea), min(params.top_edges, eb)
    return ea * eb


def test_box_box_candidates(engine):
    w = synth.make_config(1, 24)
    check_candidates(engine, w, engine.params(), range(w.n_pairs), "box-box")


def test_hull_vs_primitive_candidates(engine):
    w = synth.make_config(2, 24)
    check_candidates(engine, w, engine.params(), range(w.n_pairs), "hull vs primitive")


@pytest.mark.parametrize("tau", [1e-3, 1e-1])
def test_mixed_candidates_other_tau(engine, tau):
    w = synth.config_mixed(n=12, seed=21)
    w.tau[:] = tau
    check_candidates(engine, w, engine.params(), range(w.n_pairs), f"mixed tau={tau}")


def test_preselected_candidates(engine):
    w = synth.make_config(2, 12)
    params = engine.params(top_verts=6, top_edges=5)
    check_candidates(engine, w, params, range(w.n_pairs), "pre-selected")


def test_vertex_only_candidates(engine):
    w = synth.make_config(2, 12)
    params = engine.params(flags=1, K=4)
    check_candidates(engine, w, params, range(w.n_pairs), "vertex contacts only")


def test_offsets_checked(engine):
    """Offsets that do not match a pair's candidate count write nothing for that pair and
    are reported by cm_check_device_error."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.make_config(1, 4)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params()
    off = api.cm_candidate_offsets(engine.ctx, pg.cpu().numpy(), params)
    assert off[-1] == 4 * (16 + 2 * 144)
    bad = off.copy()
    bad[2:] += 1                                 # pair 1 one row too long
    cand = torch.full((int(bad[-1]), 8), 7.0, device="cuda")
    out = torch.empty((4, params.K, 8), device="cuda")
    api.cm_contact_manifold_fwd_dump(engine.ctx, pg, poses, dims, tau, params, out, cand,
                                     torch.as_tensor(bad, device="cuda"))
    with pytest.raises(api.CMError, match="candidate offsets"):
        engine.check()
    c = cand.cpu().numpy()
    assert (c[bad[1]:bad[2]] == 7.0).all()       # pair 1 untouched
    assert not (c[bad[0]:bad[1]] == 7.0).all()   # pair 0 written
