"""The oracle's autograd gradients on the widened paths against central finite differences
(step 1e-6, relative 1e-3 of the largest component): soft pre-selection of vertices and
edges (Sec. IV-A, Supplement B), smooth unions of superquadrics (Sec. IV-B, IV-B1) and
sphere-traced E-E witnesses (Supplement).  A detached or hard step anywhere on these
paths shows up as a gradient that differs from the differences."""
import numpy as np
import pytest
import torch

import synth
from oracle.manifold import Params, pair_manifold
from oracle.preselect import pair_manifold_preselect

F = torch.float64


def t(x):
    return torch.as_tensor(np.asarray(x), dtype=F)


def fd_vs_autograd(f, pose, dims, seed, used=slice(None)):
    """f(pose (14,), dims (6,)) -> (K, 8) tensor.  Returns (autograd, central differences)
    of sum(f * g) for a seeded g, over the entries ``used`` of (pose, dims)."""
    x = np.concatenate([pose, dims]).astype(np.float64)
    xt = t(x).requires_grad_(True)
    out = f(xt[:14], xt[14:])
    g = t(np.random.default_rng(seed).normal(size=tuple(out.shape)))
    (grad,) = torch.autograd.grad(out, xt, g)

    def loss(v):
        with torch.no_grad():
            return float((f(t(v[:14]), t(v[14:])) * g).sum())
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        fd[i] = (loss(x + e) - loss(x - e)) / (2 * h)
    return grad.numpy()[used], fd[used]


def check(grad, fd):
    assert np.isfinite(grad).all()
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(grad - fd).max() <= 1e-3 * scale + 1e-7, (np.abs(grad - fd).max(), scale)


@pytest.mark.parametrize("i", [0, 3])
def test_preselection_gradient(i):
    w = synth.config_hull_vs_primitive(n=4, seed=17, n_points=(12, 24))
    ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
    p = Params(K=4)
    f = lambda pose, dims: pair_manifold_preselect(ga, gb, pose, dims, float(w.tau[i]), p,  # noqa: E731
                                                   top_verts=4, top_edges=4)
    check(*fd_vs_autograd(f, w.poses[i], w.dims[i], seed=i, used=np.r_[0:14, 17:20]))


def test_superquadric_union_gradient():
    w = synth.config_sq_union(n=2, n_prims=3, pool=2, seed=23)
    ga, gb = w.geoms[w.pair_geoms[0, 0]], w.geoms[w.pair_geoms[0, 1]]
    f = lambda pose, dims: pair_manifold(ga, gb, pose, dims, float(w.tau[0]), Params(K=4))  # noqa: E731
    check(*fd_vs_autograd(f, w.poses[0], w.dims[0], seed=5, used=slice(0, 14)))


def test_sphere_traced_witness_gradient():
    w = synth.make_config(1, 3)
    box = w.geoms[w.pair_geoms[1, 0]]
    f = lambda pose, dims: pair_manifold(box, box, pose, dims, float(w.tau[1]),  # noqa: E731
                                         Params(K=4, trace_iters=2))
    check(*fd_vs_autograd(f, w.poses[1], w.dims[1], seed=6))
