"""Adjoint kernel against the FP64 oracle's autograd gradient and FP64 central finite
differences, through the C ABI and through the torch.autograd wrapper.  Both ways
of calling the adjoint are held to the oracle: recomputing the forward inside the
call ("recompute") and reading the forward's per-pair records ("records")."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _parity import check_grad

pytestmark = pytest.mark.gpu
REL = 1e-3        # relative to the largest gradient component of each pair


@pytest.fixture(scope="module")
def engine():
    from paper_2602_20304_gb300.engine import Engine
    e = Engine(0)
    yield e
    e.close()


def gpu_grad(engine, w, grad_out, path="recompute", **pkw):
    from paper_2602_20304_gb300.engine import workload_tensors
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params(**pkw)
    go = torch.as_tensor(grad_out, dtype=torch.float32, device="cuda").contiguous()
    saved = engine.forward_save(pg, poses, dims, tau, params)[1] if path == "records" else None
    gp, gd = engine.backward(pg, poses, dims, tau, go, params, saved=saved)
    torch.cuda.synchronize()
    engine.check()
    return gp.cpu().numpy().astype(np.float64), gd.cpu().numpy().astype(np.float64), params


def rel_errors(got, ref):
    scale = np.abs(ref).max(axis=1)
    return np.abs(got - ref).max(axis=1) / np.maximum(scale, 1e-12)


def check_against_oracle(engine, w, grad_out, path="recompute", **pkw):
    gp, gd, params = gpu_grad(engine, w, grad_out, path, **pkw)
    return check_grad(np.concatenate([gp, gd], 1), w, params, grad_out, what="gradients")["max_rel"]


def test_box_vs_hull_weighted_distance_loss(engine):
    """Loss = sum_k w_k d_k over 64 box vs 32-point-hull pairs: gradients w.r.t. both poses
    and the box dims."""
    w = synth.make_config(3, 64)
    out_grad = np.zeros((w.n_pairs, 8, 8))
    # d(sum w d)/d out = (0, 0, 0, w, 0, 0, 0, d): needs the forward values
    fwd = oracle.batch_manifold(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau)
    out_grad[..., 3] = fwd[..., 7]
    out_grad[..., 7] = fwd[..., 3]
    print("box-vs-hull32 grad rel", check_against_oracle(engine, w, out_grad))


PATHS = ["recompute", "records"]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("cfg,n", [(1, 48), (2, 48)])
def test_random_upstream(engine, cfg, n, path):
    w = synth.make_config(cfg, n)
    g = np.random.default_rng(cfg).normal(size=(w.n_pairs, 8, 8))
    print(f"config {cfg} {path} grad rel", check_against_oracle(engine, w, g, path))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("tau", [1e-3, 1e-2, 1e-1])
def test_mixed_kinds_and_tau(engine, tau, path):
    w = synth.config_mixed(n=24, seed=5)
    w.tau[:] = tau
    g = np.random.default_rng(7).normal(size=(w.n_pairs, 8, 8))
    print(f"mixed tau={tau} {path} grad rel", check_against_oracle(engine, w, g, path))


@pytest.mark.parametrize("path", PATHS)
def test_hull_vs_hull(engine, path):
    """Both bodies hulls (8..64 points each): the adjoint takes both hulls' plane
    reverses (value at the other witness, Hessian-vector product at its own)."""
    w = synth.config_hull_vs_hull(n=24, tau=1e-2)
    g = np.random.default_rng(11).normal(size=(w.n_pairs, 8, 8))
    print(f"hull-vs-hull {path} grad rel", check_against_oracle(engine, w, g, path))


@pytest.mark.parametrize("path", PATHS)
def test_vertex_contacts_only(engine, path):
    w = synth.make_config(2, 32)
    g = np.random.default_rng(3).normal(size=(w.n_pairs, 4, 8))
    check_against_oracle(engine, w, g, path, flags=1, K=4)


def test_records_match_recompute(engine):
    """The two ways of calling the adjoint agree pair by pair (to the rounding of the
    atomically summed adjoints and of the forward's reductions)."""
    w = synth.config_mixed(n=64, seed=9)
    g = np.random.default_rng(5).normal(size=(w.n_pairs, 8, 8))
    a = np.concatenate(gpu_grad(engine, w, g, "recompute")[:2], 1)
    b = np.concatenate(gpu_grad(engine, w, g, "records")[:2], 1)
    rel = rel_errors(b, a)
    print("records vs recompute, worst relative", rel.max())
    assert rel.max() <= 1e-3


def test_saved_stride_checked(engine):
    """A record buffer narrower than cm_saved_stride is refused by both calls."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import workload_tensors
    w = synth.make_config(2, 8)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    params = engine.params()
    stride = api.cm_saved_stride(engine.ctx, params)
    assert stride >= 11 * params.K
    narrow = torch.empty((w.n_pairs, stride - 4), dtype=torch.float32, device="cuda")
    out = torch.empty((w.n_pairs, params.K, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(api.CMError):
        api.cm_contact_manifold_fwd_save(engine.ctx, pg, poses, dims, tau, params, out, narrow)
    go = torch.zeros_like(out)
    gp, gd = torch.empty_like(poses), torch.empty_like(dims)
    with pytest.raises(api.CMError):
        api.cm_contact_manifold_bwd_saved(engine.ctx, pg, poses, dims, tau, params, narrow, go, gp, gd)


def test_against_fp64_central_differences(engine):
    """GPU adjoint vs central differences (step 1e-6) of the FP64 oracle."""
    w = synth.make_config(3, 6)
    rng = np.random.default_rng(11)
    g = rng.normal(size=(w.n_pairs, 8, 8))
    gp, gd, params = gpu_grad(engine, w, g)
    h = 1e-6
    for i in range(w.n_pairs):
        x = np.concatenate([w.poses[i], w.dims[i]]).astype(np.float64)
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]

        def L(v):
            with torch.no_grad():
                o = oracle.pair_manifold(ga, gb, torch.tensor(v[:14]), torch.tensor(v[14:]),
                                         float(w.tau[i]))
            return float((o.numpy() * g[i]).sum())
        fd = np.array([(L(x + h * e) - L(x - h * e)) / (2 * h) for e in np.eye(20)])
        got = np.concatenate([gp[i], gd[i]])
        keep = np.r_[0:17]                       # B is a hull: its dims do not enter
        assert np.abs(got[keep] - fd[keep]).max() <= REL * np.abs(fd[keep]).max() + 1e-6, i


def test_autograd_wrapper(engine):
    from paper_2602_20304_gb300.engine import contact_manifold, workload_tensors
    w = synth.make_config(1, 16)
    ids = engine.add_geometries(w.geoms)
    pg, poses, dims, tau = workload_tensors(w, id_map=ids)
    poses = poses.clone().requires_grad_(True)
    dims = dims.clone().requires_grad_(True)
    out = contact_manifold(engine, pg, poses, dims, tau)
    loss = (out[..., 3] * out[..., 7]).sum()
    gp, gd = torch.autograd.grad(loss, (poses, dims))
    go = torch.zeros_like(out)
    go[..., 3] = out[..., 7].detach()
    go[..., 7] = out[..., 3].detach()
    rp, rd = engine.backward(pg, poses.detach(), dims.detach(), tau, go)
    # the adjoint sums with atomics, so two launches agree to rounding, not bitwise
    assert torch.allclose(gp, rp, rtol=1e-4, atol=1e-6) and torch.allclose(gd, rd, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("pkw", [dict(top_verts=6, top_edges=5), dict(trace_iters=3), dict(K=16),
                                 dict(flags=1, K=4), dict(flags=2, K=4)],
                         ids=["preselect", "trace", "K16", "vertex-only", "one-sided"])
def test_records_on_every_path(engine, pkw):
    """The record-driven adjoint on pre-selection, sphere tracing, the K <= 16 builds and the
    simplified modes: the same gradients as the adjoint that recomputes the forward, and the
    oracle's on a sample of the pairs."""
    w = synth.make_config(2, 24)
    K = pkw.get("K", 8)
    g = np.random.default_rng(17).normal(size=(w.n_pairs, K, 8))
    a = np.concatenate(gpu_grad(engine, w, g, "recompute", **pkw)[:2], 1)
    got, gd, params = gpu_grad(engine, w, g, "records", **pkw)
    b = np.concatenate([got, gd], 1)
    rel = rel_errors(b, a)
    print(pkw, "records vs recompute, worst relative", rel.max())
    assert rel.max() <= 1e-3
    idx = np.arange(0, w.n_pairs, 3)
    check_grad(b[idx], w, params, g[idx], idx, what=f"records {pkw}")
