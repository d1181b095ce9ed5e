"""The CUDA path against the stored FP64 oracle case (tests/golden/oracle_small.json),
forward and adjoint, through the C ABI; no oracle run at test time."""
import os
import sys

import numpy as np
import pytest
import torch

import synth
from _parity import BOUND_FACTOR, SLICES, TOL, pair_errors

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

pytestmark = pytest.mark.gpu
REL = 1e-3        # gradient error relative to the largest component of each pair


def test_forward_and_adjoint_match_stored_oracle_case():
    from paper_2602_20304_gb300.engine import Engine, workload_tensors
    g = make_golden.load()
    w = synth.Workload("golden", g["geoms"], g["pair_geoms"], g["poses"], g["dims"], g["tau"])
    eng = Engine(0)
    try:
        ids = eng.add_geometries(w.geoms)
        pg, poses, dims, tau = workload_tensors(w, id_map=ids)
        sp = g["params"]
        params = eng.params(K=sp["K"])
        for k in ("w_reg", "eps_clip", "eps_min", "eps_comp", "flags"):
            assert abs(float(getattr(params, k)) - sp[k]) < 1e-7, k
        out = eng.forward(pg, poses, dims, tau, params)
        torch.cuda.synchronize()
        eng.check()
        o = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(o).all()
        e = pair_errors(o, g["manifold"])
        bound = np.maximum(np.array([TOL[k] for k in SLICES]), BOUND_FACTOR * g["spread_fwd"])
        print("stored case: pairs within TOL", float((e <= np.array([TOL[k] for k in SLICES])).all(1).mean()),
              "largest error / bound", float((e / bound).max()))
        assert (e <= bound).all(), (e / bound).max(1)
        go = torch.as_tensor(g["grad_out"], device="cuda").contiguous()
        gp, gd = eng.backward(pg, poses, dims, tau, go, params)
        torch.cuda.synchronize()
        eng.check()
        got = np.concatenate([gp.cpu().numpy(), gd.cpu().numpy()], 1).astype(np.float64)
        ref = np.concatenate([g["grad_poses"], g["grad_dims"]], 1)
        assert np.isfinite(got).all()
        err = np.abs(got - ref).max(1)
        bound = np.maximum(REL * np.abs(ref).max(1), BOUND_FACTOR * g["spread_grad"])
        assert (err <= bound).all(), err / bound
    finally:
        eng.close()
