"""Pins of the oracle's whole manifold: invariances, SoftSort limits, a closed-form
resting-box case and the autograd gradient against central finite differences."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.manifold import Params, pair_candidates, pair_manifold, soft_topk_reduce

F = torch.float64


def t(x):
    return torch.as_tensor(np.asarray(x), dtype=F)


def swap_pose(p):
    return np.concatenate([p[7:], p[:7]])


def swap_dims(d):
    return np.concatenate([d[3:], d[:3]])


def _pairs():
    w1 = synth.make_config(1, 6)
    w2 = synth.config_hull_vs_primitive(n=8, seed=7, n_points=(8, 20))
    out = []
    for w in (w1, w2):
        for i in range(w.n_pairs):
            ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
            out.append((ga, gb, w.poses[i].astype(np.float64), w.dims[i].astype(np.float64),
                        float(w.tau[i])))
    return out


PAIRS = _pairs()


@pytest.mark.parametrize("k", range(len(PAIRS)))
def test_swap_symmetry(k):
    """manifold(A, B) == manifold(B, A): the candidate multiset is the same once witness
    roles and row/column nearest-neighbour softmaxes are exchanged."""
    ga, gb, pose, dims, tau = PAIRS[k]
    m1 = pair_manifold(ga, gb, t(pose), t(dims), tau).numpy()
    m2 = pair_manifold(gb, ga, t(swap_pose(pose)), t(swap_dims(dims)), tau).numpy()
    assert np.abs(m1 - m2).max() < 1e-10


@pytest.mark.parametrize("k", [0, 3, 7, 10])
def test_rigid_motion_covariance(k):
    ga, gb, pose, dims, tau = PAIRS[k]
    rng = np.random.default_rng(k)
    q0 = synth.random_quaternions(rng, 1)[0]
    R0 = oracle.quat_to_rot(t(q0)).numpy()
    t0 = rng.uniform(-2, 2, 3)

    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    moved = pose.copy()
    for o in (0, 7):
        moved[o:o + 4] = qmul(q0, pose[o:o + 4])
        moved[o + 4:o + 7] = R0 @ pose[o + 4:o + 7] + t0
    m1 = pair_manifold(ga, gb, t(pose), t(dims), tau).numpy()
    m2 = pair_manifold(ga, gb, t(moved), t(dims), tau).numpy()
    assert np.abs(m2[:, 3] - m1[:, 3]).max() < 1e-9
    assert np.abs(m2[:, 7] - m1[:, 7]).max() < 1e-9
    assert np.abs(m2[:, :3] - (m1[:, :3] @ R0.T + t0)).max() < 1e-9
    assert np.abs(m2[:, 4:7] - m1[:, 4:7] @ R0.T).max() < 1e-9


def test_softsort_limits():
    rng = np.random.default_rng(3)
    cand = t(rng.normal(size=(40, 8)))
    cand[:, 7] = t(rng.uniform(0.1, 1.0, 40))
    s = -(cand[:, 7] * cand[:, 3]).numpy()
    order = np.argsort(-s)
    hard = soft_topk_reduce(cand, 1e-9, 8).numpy()
    assert np.abs(hard - cand.numpy()[order[:8]]).max() < 1e-12
    ones = cand.clone()
    ones[:, 0] = 1.0
    assert np.abs(soft_topk_reduce(ones, 0.1, 8).numpy()[:, 0] - 1.0).max() < 1e-14
    eq = cand.clone()
    eq[:, 3] = -0.2
    eq[:, 7] = 0.5                              # all scores equal -> uniform rows
    out = soft_topk_reduce(eq, 0.05, 8).numpy()
    assert np.abs(out - eq.numpy().mean(0)).max() < 1e-14


def test_softsort_two_score_levels_closed_form():
    """Sec. III SoftSort on two score levels a gap tau ln 3 apart: one candidate x0 on top,
    three (x1..x3) below.  Row 1 sits on the top score: weights 1 and e^{-ln 3} = 1/3 each,
    normalised to 1/2 and 1/6.  Row 2 sits on the lower level: x0 gets 1/3 against 1 for
    each of the others, i.e. 1/10 and 3/10.  (Without the absolute value in the logits
    row 2 would weigh x0 by 3 instead of 1/3.)"""
    tau = 0.05
    rng = np.random.default_rng(11)
    cand = t(rng.normal(size=(4, 8)))
    cand[:, 7] = 1.0
    cand[0, 3] = -0.5
    cand[1:, 3] = -0.5 + tau * np.log(3.0)
    out = soft_topk_reduce(cand, tau, 2).numpy()
    x = cand.numpy()
    np.testing.assert_allclose(out[0], x[0] / 2 + x[1:].sum(0) / 6, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out[1], x[0] / 10 + 3 * x[1:].sum(0) / 10, rtol=0, atol=1e-13)


def test_softsort_ignores_candidate_order():
    """The reduction depends on the candidate set, not on the order of the rows."""
    rng = np.random.default_rng(12)
    cand = t(rng.normal(size=(50, 8)))
    cand[:, 7] = t(rng.uniform(0.0, 1.0, 50))
    perm = torch.as_tensor(rng.permutation(50))
    for tau in (1e-3, 1e-2, 1e-1):
        a = soft_topk_reduce(cand, tau, 8).numpy()
        b = soft_topk_reduce(cand[perm], tau, 8).numpy()
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


def test_resting_box_closed_form():
    """Small cube (h = 0.3) resting axis-aligned on a larger one (h = 0.5) with depth delta.
    As tau -> 0 its four bottom vertices read d = -delta with normal +z and activity 1."""
    box = synth.primitive_geometry(synth.KIND_BOX)
    delta, tau = 0.05, 1e-4
    pose = np.array([1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0.8 - delta], dtype=np.float64)
    dims = np.array([0.5, 0.5, 0.5, 0.3, 0.3, 0.3])
    cand = pair_candidates(box, box, t(pose), t(dims), tau).numpy()
    vb = cand[8:16]                              # B's vertices against A
    bottom = vb[vb[:, 2] < 0.6]
    assert len(bottom) == 4
    assert np.abs(bottom[:, 3] + delta).max() < 1e-9
    assert np.abs(bottom[:, 4:7] - [0, 0, 1 / np.sqrt(1 + tau)]).max() < 1e-9
    assert np.abs(bottom[:, 7] - 1).max() < 1e-9
    # with V-S contacts only (the "no E-E" simplification) the four bottom vertices tie for
    # the largest score and the first contact point is their centre
    nov = Params(no_ee=True)
    cv = pair_candidates(box, box, t(pose), t(dims), tau, nov).numpy()
    s = -cv[:, 7] * cv[:, 3]
    assert np.sort(s)[-5] < delta - 1e-3
    m = pair_manifold(box, box, t(pose), t(dims), tau, nov).numpy()
    assert np.abs(m[0, :3] - [0, 0, 0.5 - delta]).max() < 1e-9
    assert abs(m[0, 3] + delta) < 1e-9 and abs(m[0, 7] - 1) < 1e-9
    # with E-E contacts the parallel bottom/top edge pairs add witnesses at the line-line
    # distance sqrt(0.2^2 + delta^2) with clashing indicator 1/2 (orthogonal corner normals)
    s = -cand[:, 7] * cand[:, 3]
    top = cand[np.argsort(-s)[:4]]
    assert np.abs(top[:, 3] + np.hypot(0.2, delta)).max() < 1e-6


def _fd_check(ga, gb, pose, dims, tau, seed):
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(8, 8))
    x = np.concatenate([pose, dims])

    def loss(v):
        with torch.no_grad():
            return float((pair_manifold(ga, gb, t(v[:14]), t(v[14:]), tau).numpy() * g).sum())
    xt = t(x).requires_grad_(True)
    out = pair_manifold(ga, gb, xt[:14], xt[14:], tau)
    (grad,) = torch.autograd.grad(out, xt, t(g))
    grad = grad.numpy()
    h = 1e-6
    fd = np.zeros_like(x)
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        fd[i] = (loss(x + e) - loss(x - e)) / (2 * h)
    return grad, fd


@pytest.mark.parametrize("k", [1, 2, 6, 9])
def test_gradient_vs_central_fd(k):
    ga, gb, pose, dims, tau = PAIRS[k]
    grad, fd = _fd_check(ga, gb, pose, dims, tau, seed=k)
    if ga.kind == synth.KIND_HULL:
        grad, fd = grad[np.r_[0:14, 17:20]], fd[np.r_[0:14, 17:20]]   # hull dims are unused
    scale = np.abs(fd).max()
    assert np.abs(grad - fd).max() <= 1e-3 * scale + 1e-7
