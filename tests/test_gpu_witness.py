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


def test_vertex_face_witness_batch():
    from paper_2602_20304_gb300 import api
    rng = np.random.default_rng(2)
    n = 200_000
    q = rng.uniform(0, 1, size=(n, 12)).astype(np.float32)
    t = torch.from_numpy(q.astype(np.float64))
    area = torch.linalg.vector_norm(torch.cross(t[:, 6:9] - t[:, 3:6], t[:, 9:12] - t[:, 3:6], dim=1), dim=1)
    # the plane normal of a thin triangle carries FP32 error / |cross|: sliver triangles
    # (|(t1 - t0) x (t2 - t0)| < 0.05, 0.8% of the queries) are outside the fixed tolerance
    keep = (area > 5e-2).numpy()
    out = torch.empty((n, 4), device="cuda")
    api.cm_vf_witness_batch(torch.from_numpy(q).cuda(), api.cm_default_params(), out)
    got = out.cpu().numpy().astype(np.float64)
    w, inside = oracle.vf_witness(t[:, 0:3], t[:, 3:6], t[:, 6:9], t[:, 9:12])
    assert np.abs(got[keep, 0:3] - w.numpy()[keep]).max() < 1e-5
    assert np.abs(got[keep, 3] - inside.numpy()[keep]).max() < 1e-5


def test_empty_and_misaligned():
    from paper_2602_20304_gb300 import api
    p = api.cm_default_params()
    api.cm_ee_witness_batch(torch.empty((0, 12), device="cuda"), p, torch.empty((0, 8), device="cuda"))
    buf = torch.empty(12 * 4 + 1, device="cuda")
    with pytest.raises(api.CMError):
        api.cm_ee_witness_batch(buf[1:].view(4, 12), p, torch.empty((4, 8), device="cuda"))
