"""Soft top-K pre-selection of vertices and edges (with the safeguard) against the oracle."""
import numpy as np
import pytest
import torch

import synth
from _parity import TOL, assert_close, oracle_forward

# Pre-selection adds one more SoftSort, over FP32 vertex / edge depths at temperature
# tau: its weights carry the depth rounding times 1/tau into the selected positions
# before the contacts are generated, so these tests allow twice the fixed tolerance.
TOL_SEL = {k: 2 * v for k, v in TOL.items()}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def engine():
    from paper_2602_20304_gb300.engine import Engine
    e = Engine(0)
    yield e
    e.close()


def run(engine, w, **pkw):
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params(**pkw)
    out = engine.forward(pg, poses, dims, tau, params)
    torch.cuda.synchronize()
    engine.check()
    return out.cpu().numpy().astype(np.float64), params


@pytest.mark.parametrize("tv,te", [(0, 8), (8, 8), (16, 16), (4, 0)])
def test_preselection_matches_oracle(engine, tv, te):
    w = synth.make_config(2, 48)
    gpu, params = run(engine, w, top_verts=tv, top_edges=te)
    print(f"top_verts={tv} top_edges={te}",
          assert_close(gpu, oracle_forward(w, params), tol=TOL_SEL, what=f"preselect {tv}/{te}"))


def test_preselection_on_boxes(engine):
    w = synth.make_config(1, 64)
    gpu, params = run(engine, w, top_edges=4)
    assert_close(gpu, oracle_forward(w, params), tol=TOL_SEL, what="box-box preselect")


def test_adjoint_rejects_preselection(engine):
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.make_config(1, 4)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    with pytest.raises(api.CMError):
        engine.backward(pg, poses, dims, tau, torch.zeros((4, 8, 8), device="cuda"),
                        engine.params(top_edges=4))
