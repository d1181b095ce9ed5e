"""Soft top-K pre-selection of vertices and edges (with the safeguard) against the oracle."""
import numpy as np
import pytest
import torch

import synth
from _parity import check_forward, check_grad

# Pre-selection adds one more SoftSort, over FP32 vertex / edge depths at temperature
# tau: its weights carry the depth rounding times 1/tau into the selected positions
# before the contacts are generated.  Pairs where that matters are held to their own
# one-ulp conditioning bound (tests/_parity.py), the others to the fixed tolerance.

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
    check_forward(gpu, w, params, what=f"preselect {tv}/{te}")


def test_preselection_on_boxes(engine):
    w = synth.make_config(1, 64)
    gpu, params = run(engine, w, top_edges=4)
    check_forward(gpu, w, params, what="box-box preselect")


@pytest.mark.parametrize("cfg,n,tv,te", [(1, 24, 0, 4), (1, 24, 4, 4), (2, 16, 0, 8), (2, 16, 8, 8),
                                         (3, 12, 4, 0), ("sq", 6, 0, 5)])
def test_preselection_adjoint(engine, cfg, n, tv, te):
    """The adjoint through the soft selection (scores from vertex depths), the safeguard
    and the selected contacts against the oracle's autograd.  Through the selection the
    gradient is a 1/tau-scaled difference of neighbouring items' score gradients, which
    cancels and so amplifies rounding; each pair is held to 1e-3 of its largest component
    or, where its inputs' one-ulp rounding alone moves the oracle's gradient more, to its
    own conditioning bound (tests/_parity.py)."""
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.config_sq_union(n=n, n_prims=5, pool=3) if cfg == "sq" else synth.make_config(cfg, n)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params(top_verts=tv, top_edges=te)
    g = np.random.default_rng(tv + te).normal(size=(n, params.K, 8))
    gp, gd = engine.backward(pg, poses, dims, tau, torch.as_tensor(g, dtype=torch.float32, device="cuda"), params)
    torch.cuda.synchronize()
    engine.check()
    got = np.concatenate([gp.cpu().numpy(), gd.cpu().numpy()], 1).astype(np.float64)
    check_grad(got, w, params, g, what=f"preselect {cfg} {tv}/{te} gradients")
