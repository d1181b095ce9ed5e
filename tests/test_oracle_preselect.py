"""Pins of the oracle's soft top-K pre-selection (Sec. IV-A; Supplement B)."""
import numpy as np
import pytest
import torch

import synth
from oracle.manifold import Params, pair_manifold
from oracle.preselect import pair_manifold_preselect, soft_select

F = torch.float64


def t(x):
    return torch.as_tensor(np.asarray(x), dtype=F)


def test_soft_select_hard_limit_and_rows():
    rng = np.random.default_rng(0)
    score = t(rng.normal(size=30))
    vals = t(rng.normal(size=(30, 4)))
    sel, gamma = soft_select(score, vals, 5, 1e-9)
    order = np.argsort(-score.numpy())[:5]
    assert np.abs(sel.numpy() - vals.numpy()[order]).max() < 1e-12
    _, g = soft_select(score, vals, 5, 0.3)
    assert torch.allclose(g.sum(1), torch.ones(5, dtype=F), atol=1e-14)


def _pairs():
    w1 = synth.make_config(1, 3)
    w2 = synth.config_hull_vs_primitive(n=4, seed=11, n_points=(10, 16))
    out = []
    for w in (w1, w2):
        for i in range(w.n_pairs):
            out.append((w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]], w.poses[i].astype(np.float64),
                        w.dims[i].astype(np.float64), float(w.tau[i])))
    return out


@pytest.mark.parametrize("k", range(7))
def test_selecting_everything_in_the_hard_limit_is_the_plain_manifold(k):
    ga, gb, pose, dims, tau = _pairs()[k]
    p = Params()
    plain = pair_manifold(ga, gb, t(pose), t(dims), tau, p).numpy()
    sel = pair_manifold_preselect(ga, gb, t(pose), t(dims), tau, p, top_verts=256, top_edges=768,
                                  safeguard=False, tau_sel=1e-12).numpy()
    assert np.abs(plain - sel).max() < 1e-9


def test_deepest_edges_are_selected():
    """A small cube resting on a large one with depth delta: in the hard limit the two
    selected edges of the small cube are bottom edges (both corners at depth delta)."""
    box = synth.primitive_geometry(synth.KIND_BOX)
    delta = 0.05
    pose = np.array([1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0.8 - delta])
    dims = np.array([0.5, 0.5, 0.5, 0.3, 0.3, 0.3])
    from oracle.manifold import _Body
    from oracle.preselect import soft_select as ss
    B = _Body(box, t(pose[7:]), t(dims[3:]), 1e-4)
    A = _Body(box, t(pose[:7]), t(dims[:3]), 1e-4)
    m, _ = A.sdf(B.verts)
    me = 0.5 * (m[B.edges[:, 0]] + m[B.edges[:, 1]])
    sel, _ = ss(-me, torch.cat([B.verts[B.edges[:, 0]], B.verts[B.edges[:, 1]]], 1), 2, 1e-9)
    assert np.abs(sel[:, 2].numpy() - (0.5 - delta)).max() < 1e-9 and np.abs(sel[:, 5].numpy() - (0.5 - delta)).max() < 1e-9
