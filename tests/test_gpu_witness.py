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
