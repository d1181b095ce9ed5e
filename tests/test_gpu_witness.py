"""Batched witness-point routines (the witness-point throughput setting) against the oracle:
queries uniform in the unit cube, as in the paper's experiment."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def test_edge_edge_witness_batch():
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(1)
    n = 200_000
    q = rng.uniform(0, 1, size=(n, 12)).astype(np.float32)
    out = torch.empty((n, 8), device="cuda")
    api.cm_ee_witness_batch(torch.from_numpy(q).cuda(), api.cm_default_params(), out)
    got = out.cpu().numpy().astype(np.float64)
    t = torch.from_numpy(q.astype(np.float64))
    e1, e2, _, _, con = oracle.ee_witness(t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12])
    assert np.abs(got[:, 0:3] - e1.numpy()).max() < 1e-5
    assert np.abs(got[:, 3:6] - e2.numpy()).max() < 1e-5
    assert np.abs(got[:, 6] - con.numpy()).max() < 1e-5
    assert np.abs(got[:, 7] - torch.linalg.vector_norm(e1 - e2, dim=1).numpy()).max() < 1e-5


def test_edge_edge_witness_near_parallel():
    """Edge pairs 1e-6 .. 1e-3 rad from parallel, the subset where the 2x2 solve is
    worst conditioned (Q^T Q is singular without the L2 term): the FP32 kernel holds the
    same 1e-5 as on generic queries, so the solve needs no FP64."""
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(5)
    n = 200_000
    unit = lambda v: v / np.linalg.norm(v, axis=1, keepdims=True)  # noqa: E731
    u = unit(rng.standard_normal((n, 3)))
    perp = unit(np.cross(u, rng.standard_normal((n, 3))))
    th = 10.0 ** rng.uniform(-6, -3, n)
    u2 = np.cos(th)[:, None] * u + np.sin(th)[:, None] * perp
    a0 = rng.uniform(0, 1, (n, 3))
    b0 = a0 + rng.uniform(-0.3, 0.3, (n, 3))
    q = np.concatenate([a0, a0 + rng.uniform(0.2, 1, (n, 1)) * u,
                        b0, b0 + rng.uniform(0.2, 1, (n, 1)) * u2], 1).astype(np.float32)
    out = torch.empty((n, 8), device="cuda")
    api.cm_ee_witness_batch(torch.from_numpy(q).cuda(), api.cm_default_params(), out)
    got = out.cpu().numpy().astype(np.float64)
    t = torch.from_numpy(q.astype(np.float64))
    e1, e2, _, _, con = oracle.ee_witness(t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12])
    err = [np.abs(got[:, 0:3] - e1.numpy()).max(), np.abs(got[:, 3:6] - e2.numpy()).max(),
           np.abs(got[:, 6] - con.numpy()).max(),
           np.abs(got[:, 7] - torch.linalg.vector_norm(e1 - e2, dim=1).numpy()).max()]
    print("near-parallel e1, e2, con, dbar max errors", err)
    assert max(err) < 1e-5, err


def test_vertex_face_witness_batch():
    """V-F witnesses of 2e5 random queries against the oracle: within 1e-5, or for the
    queries that miss it (sliver triangles, whose plane normal carries FP32 error /
    |(t1 - t0) x (t2 - t0)|) within 16 times the oracle's own move when the query's twelve
    FP32 coordinates move by one ulp (four draws; the per-pair bar of tests/_parity.py)."""
    from _parity import BOUND_FACTOR, ULP_DRAWS, _ulp
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(2)
    n = 200_000
    q = rng.uniform(0, 1, size=(n, 12)).astype(np.float32)
    out = torch.empty((n, 4), device="cuda")
    api.cm_vf_witness_batch(torch.from_numpy(q).cuda(), api.cm_default_params(), out)
    got = out.cpu().numpy().astype(np.float64)

    def ref_of(qq):
        t = torch.from_numpy(qq.astype(np.float64))
        w, inside = oracle.vf_witness(t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12])
        return np.concatenate([w.numpy(), inside.numpy()[:, None]], 1)
    ref = ref_of(q)
    err = np.abs(got - ref).max(1)
    over = np.nonzero(err > 1e-5)[0]
    print("V-F queries within 1e-5:", 1 - len(over) / n)
    assert len(over) / n < 0.05
    spread = np.zeros(len(over))
    draw = np.random.default_rng(3)
    for _ in range(ULP_DRAWS):
        spread = np.maximum(spread, np.abs(ref_of(_ulp(q[over], draw)) - ref[over]).max(1))
    ratio = err[over] / np.maximum(spread, 1e-300)
    print("largest error / one-ulp spread among them:", float(ratio.max()) if len(over) else 0.0)
    assert (err[over] <= BOUND_FACTOR * spread).all(), (int(over[np.argmax(ratio)]), float(ratio.max()))


def test_empty_and_misaligned():
    from paper_2602_20304_gb300 import api
    p = api.cm_default_params()
    api.cm_ee_witness_batch(torch.empty((0, 12), device="cuda"), p, torch.empty((0, 8), device="cuda"))
    buf = torch.empty(12 * 4 + 1, device="cuda")
    with pytest.raises(api.CMError):
        api.cm_ee_witness_batch(buf[1:].view(4, 12), p, torch.empty((4, 8), device="cuda"))


def _hard_params():
    from paper_2602_20304_gb300 import api
    return api.cm_default_params(flags=api.CM_FLAG_HARD)


def test_edge_edge_witness_batch_hard():
    """Non-smoothed E-E routine (Ours-NS) on 2e5 unit-cube queries.  Its result is the
    minimiser of the strictly convex regularised box QP.  Where the objective is flat (near
    parallel edges, two sides' costs within FP32 resolution of each other) points far apart
    are optimal to FP32 precision, so the minimiser is not unique at that precision: what is
    unique is the optimal value.  The witnesses and their distance are held to 1e-5 for at
    least 99.9 % of the queries; every other query must give a feasible point whose FP64
    objective is within 1e-6 of the optimum.  con is 0 or 1 and must equal the oracle's
    wherever the unconstrained minimiser lies more than 1e-4 from the box's boundary."""
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(11)
    n = 200_000
    q = rng.uniform(0, 1, size=(n, 12)).astype(np.float32)
    out = torch.empty((n, 8), device="cuda")
    api.cm_ee_witness_batch(torch.from_numpy(q).cuda(), _hard_params(), out)
    got = out.cpu().numpy().astype(np.float64)
    t = torch.from_numpy(q.astype(np.float64))
    a0, a1, b0, b1 = t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12]
    e1, e2, _, _, con = oracle.ee_witness(a0, a1, b0, b1, hard=True)
    err = np.maximum(np.abs(got[:, 0:3] - e1.numpy()).max(1), np.abs(got[:, 3:6] - e2.numpy()).max(1))
    err = np.maximum(err, np.abs(got[:, 7] - torch.linalg.vector_norm(e1 - e2, dim=1).numpy()))
    over = err > 1e-5
    print("hard E-E witnesses within 1e-5:", 1 - over.mean(), "interior share", float(con.mean()))
    assert over.mean() <= 1e-3
    assert set(np.unique(got[:, 6])) <= {0.0, 1.0}
    lam = 0.01

    def objective(e1x, e2x, al1, al2):
        return ((e1x - e2x) ** 2).sum(1) + lam * ((al1 - 0.5) ** 2 + (al2 - 0.5) ** 2)
    A0, A1, B0, B1 = (x.numpy()[over] for x in (a0, a1, b0, b1))
    g1, g2 = got[over, 0:3], got[over, 3:6]
    al1 = ((g1 - A0) * (A1 - A0)).sum(1) / ((A1 - A0) ** 2).sum(1)
    al2 = ((g2 - B0) * (B1 - B0)).sum(1) / ((B1 - B0) ** 2).sum(1)
    assert (al1 > -1e-6).all() and (al1 < 1 + 1e-6).all() and (al2 > -1e-6).all() and (al2 < 1 + 1e-6).all()
    assert np.abs(g1 - (A0 + al1[:, None] * (A1 - A0))).max() < 1e-5     # on the edges
    assert np.abs(g2 - (B0 + al2[:, None] * (B1 - B0))).max() < 1e-5
    r1 = ((e1.numpy()[over] - A0) * (A1 - A0)).sum(1) / ((A1 - A0) ** 2).sum(1)
    r2 = ((e2.numpy()[over] - B0) * (B1 - B0)).sum(1) / ((B1 - B0) ** 2).sum(1)
    gap = objective(g1, g2, al1, al2) - objective(e1.numpy()[over], e2.numpy()[over], r1, r2)
    print("off-point queries:", int(over.sum()), "largest objective excess", float(gap.max()) if over.any() else 0.0)
    assert (gap <= 1e-6).all()
    # margin of the unconstrained minimiser from the box boundary, in FP64
    t1, t2, bb = a1 - a0, b0 - b1, a0 - b0
    Q11 = (t1 * t1).sum(1) + lam
    Q12 = (t1 * t2).sum(1)
    Q22 = (t2 * t2).sum(1) + lam
    c1 = (t1 * bb).sum(1) - 0.5 * lam
    c2 = (t2 * bb).sum(1) - 0.5 * lam
    det = Q11 * Q22 - Q12 * Q12
    au = torch.stack([(Q12 * c2 - Q22 * c1) / det, (Q12 * c1 - Q11 * c2) / det], 1).numpy()
    margin = np.minimum(np.abs(au), np.abs(au - 1.0)).min(1)
    clear = margin > 1e-4
    assert (got[clear, 6] == con.numpy()[clear]).all()
    assert 0.05 < con.numpy().mean() < 0.95          # both branches are exercised


def test_vertex_face_witness_batch_hard():
    """Non-smoothed V-F routine (Ours-NS): the exact closest point of the triangle, held to
    1e-5 for at least 99.9 % of the queries; every other query (the FP32 inside decision or
    edge choice taken the other way, mostly on thin triangles) must give a point on the
    triangle whose distance to the vertex is within 1e-6 of the optimal distance, the
    value that is unique.  The inside flag must equal the oracle's wherever the plane
    projection's smallest barycentric coordinate is more than 1e-4 from 0 and the oracle's
    own flag survives one-ulp moves of the query."""
    from _parity import ULP_DRAWS, _ulp
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(12)
    n = 200_000
    q = rng.uniform(0, 1, size=(n, 12)).astype(np.float32)
    out = torch.empty((n, 4), device="cuda")
    api.cm_vf_witness_batch(torch.from_numpy(q).cuda(), _hard_params(), out)
    got = out.cpu().numpy().astype(np.float64)

    def ref_of(qq):
        t = torch.from_numpy(qq.astype(np.float64))
        w, inside = oracle.vf_witness(t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12], hard=True)
        return w.numpy(), inside.numpy()
    w_ref, in_ref = ref_of(q)
    err = np.abs(got[:, 0:3] - w_ref).max(1)
    over = np.nonzero(err > 1e-5)[0]
    print("hard V-F queries within 1e-5:", 1 - len(over) / n, "inside share", float(in_ref.mean()))
    assert len(over) / n <= 1e-3
    flips = np.zeros(n, bool)
    draw = np.random.default_rng(13)
    for _ in range(ULP_DRAWS):
        flips |= ref_of(_ulp(q, draw))[1] != in_ref
    assert set(np.unique(got[:, 3])) <= {0.0, 1.0}
    qd = q[over].astype(np.float64)
    vv, T0, T1, T2 = qd[:, 0:3], qd[:, 3:6], qd[:, 6:9], qd[:, 9:12]
    pg = got[over, 0:3]
    nb_o = np.cross(T1 - T0, T2 - T0)
    a2_o = np.linalg.norm(nb_o, axis=1)
    n_o = nb_o / a2_o[:, None]
    assert (np.abs(((pg - T0) * n_o).sum(1)) < 1e-5).all()               # in the triangle's plane
    c2 = (np.cross(T1 - T0, pg - T0) * n_o).sum(1) / a2_o
    c1 = (np.cross(pg - T0, T2 - T0) * n_o).sum(1) / a2_o
    tol_b = 1e-5 / np.minimum(a2_o, 1.0)
    assert (np.minimum(np.minimum(1 - c1 - c2, c1), c2) > -tol_b).all()   # inside it
    excess = np.linalg.norm(vv - pg, axis=1) - np.linalg.norm(vv - w_ref[over], axis=1)
    print("off-point queries:", len(over), "largest distance excess", float(excess.max()) if len(over) else 0.0)
    assert (excess <= 1e-6).all()
    # smallest barycentric coordinate of the plane projection, FP64
    t = torch.from_numpy(q.astype(np.float64))
    v, t0, t1, t2 = t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12]
    nb = torch.cross(t1 - t0, t2 - t0, dim=1)
    area2 = torch.linalg.vector_norm(nb, dim=1)
    nrm = nb / area2[:, None]
    rel = v - t0
    p = rel - (rel * nrm).sum(1, keepdim=True) * nrm
    b2 = (torch.cross(t1 - t0, p, dim=1) * nrm).sum(1) / area2
    b1 = (torch.cross(p, t2 - t0, dim=1) * nrm).sum(1) / area2
    bmin = torch.minimum(torch.minimum(1.0 - b1 - b2, b1), b2).numpy()
    clear = (np.abs(bmin) > 1e-4) & ~flips
    assert (got[clear, 3] == in_ref[clear]).all()
    assert 0.05 < in_ref.mean() < 0.95


def test_hard_flag_refused_by_the_manifold():
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    import synth
    w = synth.make_config(1, 4)
    eng = Engine(0)
    try:
        ids = eng.add_geometries(w.geoms)
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        with pytest.raises(api.CMError):
            eng.forward(pg, poses, dims, tau, _hard_params())
    finally:
        eng.close()
