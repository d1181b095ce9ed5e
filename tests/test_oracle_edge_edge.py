"""Pins of the oracle's E-E witness routine (Sec. IV-D2) against brute force and closed forms."""
import numpy as np
import pytest
import torch

import oracle

F = torch.float64


def t(x):
    return torch.as_tensor(np.asarray(x), dtype=F)


def witness(a0, a1, b0, b1, **kw):
    e1, e2, al1, al2, con = oracle.ee_witness(t(a0), t(a1), t(b0), t(b1), **kw)
    return e1.numpy(), e2.numpy(), al1.numpy(), al2.numpy(), con.numpy()


def brute_force(a0, a1, b0, b1, lam, n=2001):
    """Dense grid minimisation of |e1(a1) - e2(a2)|^2 + lam |alpha - 1/2|^2 over [0, 1]^2."""
    g = np.linspace(0.0, 1.0, n)
    A1, A2 = np.meshgrid(g, g, indexing="ij")
    e1 = a0[None, None] + A1[..., None] * (a1 - a0)[None, None]
    e2 = b0[None, None] + A2[..., None] * (b1 - b0)[None, None]
    J = ((e1 - e2) ** 2).sum(-1) + lam * ((A1 - 0.5) ** 2 + (A2 - 0.5) ** 2)
    i = np.unravel_index(np.argmin(J), J.shape)
    return g[i[0]], g[i[1]], J[i]


@pytest.mark.parametrize("seed", range(12))
def test_hard_limit_matches_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    a0, a1, b0, b1 = rng.uniform(0, 1, size=(4, 3))
    lam = 0.01
    hard = dict(w_reg=lam, eps_clip=1e-7, eps_min=1e-7, eps_comp=1e-7)
    _, _, al1, al2, _ = witness(a0, a1, b0, b1, **hard)
    g1, g2, Jg = brute_force(a0, a1, b0, b1, lam)
    assert abs(al1 - g1) < 2e-3 and abs(al2 - g2) < 2e-3
    e1 = a0 + al1 * (a1 - a0)
    e2 = b0 + al2 * (b1 - b0)
    J = ((e1 - e2) ** 2).sum() + lam * ((al1 - 0.5) ** 2 + (al2 - 0.5) ** 2)
    assert J <= Jg + 1e-9                          # never worse than the grid minimum


@pytest.mark.parametrize("h", [0.1, 0.5, 2.0])
@pytest.mark.parametrize("smooth", [True, False])
def test_skew_perpendicular_closed_form(h, smooth):
    kw = {} if smooth else dict(eps_clip=1e-7, eps_min=1e-7, eps_comp=1e-7)
    e1, e2, al1, al2, _ = witness([-1, 0, 0], [1, 0, 0], [0, -1, h], [0, 1, h], **kw)
    assert abs(al1 - 0.5) < 1e-14 and abs(al2 - 0.5) < 1e-14
    assert np.abs(e1).max() < 1e-14
    assert abs(np.linalg.norm(e1 - e2) - h) < 1e-14


@pytest.mark.parametrize("s", [-0.3, 0.0, 0.2, 0.45])
def test_parallel_edges_regularised_closed_form(s):
    """Parallel unit edges one unit apart, shifted by s: the regularised minimiser is
    a1 - a2 = 2s / (2 + lam), a1 + a2 = 1 (derived by hand from the objective)."""
    lam = 0.01
    kw = dict(w_reg=lam, eps_clip=1e-8, eps_min=1e-8, eps_comp=1e-8)
    _, _, al1, al2, con = witness([0, 0, 0], [1, 0, 0], [s, 1, 0], [s + 1, 1, 0], **kw)
    u = 2 * s / (2 + lam)
    assert abs(al1 - (1 + u) / 2) < 1e-9 and abs(al2 - (1 - u) / 2) < 1e-9
    assert abs(con - 1.0) < 1e-9


@pytest.mark.parametrize("seed", range(8))
def test_swap_equivariance(seed):
    """Exchanging the two edges exchanges (alpha1, alpha2): the four side minimisers and
    their costs map onto each other only if every cost is the objective at its own point."""
    rng = np.random.default_rng(200 + seed)
    a0, a1, b0, b1 = rng.uniform(-1, 1, size=(4, 3))
    e1, e2, al1, al2, c = witness(a0, a1, b0, b1)
    f1, f2, bl1, bl2, d = witness(b0, b1, a0, a1)
    assert abs(al1 - bl2) < 1e-13 and abs(al2 - bl1) < 1e-13 and abs(c - d) < 1e-13
    assert np.abs(e1 - f2).max() < 1e-13 and np.abs(e2 - f1).max() < 1e-13


def test_interior_solution_is_unconstrained_minimiser():
    # crossing edges whose closest points are interior: con ~ 1 and alpha = -Q^-1 c
    _, _, al1, al2, con = witness([-1, 0.2, 0], [1, 0.2, 0], [0.3, -1, 0.4], [0.3, 1, 0.4],
                                  w_reg=0.0, eps_clip=1e-8, eps_min=1e-8, eps_comp=1e-8)
    assert abs(al1 - 0.65) < 1e-12 and abs(al2 - 0.6) < 1e-12 and abs(con - 1) < 1e-12


def _rotating_sweep(thetas, **kw):
    """Fig. 4 set-up: edge 2 fixed along x at y = -1.2; edge 1 of half-length 1 rotates
    about the z axis through the origin and is parallel to edge 2 at theta = pi / 2."""
    out = []
    for th in thetas:
        d = np.array([np.sin(th), np.cos(th), 0.0])
        e1, _, _, _, _ = witness(-d, d, [-2.0, -1.2, 0.0], [2.0, -1.2, 0.0], **kw)
        out.append(e1)
    return np.array(out)


def test_fig4_sweep_continuity_and_unsmoothed_jump():
    th_even = np.linspace(np.pi / 2 - 0.02, np.pi / 2 + 0.02, 400)     # skips pi / 2 itself
    hard = _rotating_sweep(th_even, w_reg=1e-12, eps_clip=1e-9, eps_min=1e-9, eps_comp=1e-9)
    jumps = np.linalg.norm(np.diff(hard, axis=0), axis=1)
    assert jumps.max() > 1.5                               # witness flips end to end
    slopes = []
    for n in (401, 1601):                                   # both grids contain pi / 2
        th = np.linspace(np.pi / 2 - 0.02, np.pi / 2 + 0.02, n)
        soft = _rotating_sweep(th)
        steps = np.linalg.norm(np.diff(soft, axis=0), axis=1)
        slopes.append(steps.max() / (th[1] - th[0]))
        assert abs(soft[n // 2, 0]) < 1e-9                  # at exact parallel: the centre
    # smoothed: the largest step shrinks with the grid (a finite Lipschitz slope) ...
    assert slopes[0] < 1e3 and abs(slopes[1] / slopes[0] - 1) < 1e-2
    # ... while the unsmoothed witness still jumps end to end on the finer grid
    th_even = np.linspace(np.pi / 2 - 0.02, np.pi / 2 + 0.02, 1600)
    hard = _rotating_sweep(th_even, w_reg=1e-12, eps_clip=1e-9, eps_min=1e-9, eps_comp=1e-9)
    assert np.linalg.norm(np.diff(hard, axis=0), axis=1).max() > 1.5


def test_crossing_penetrating_edges():
    """A unit cube A and a box B (half-extents 1, 0.5, 0.5) turned 45 degrees about x so
    that its lowest edge runs along x at height 0.5 - delta and crosses A's top edge
    x = 0.5 (along y) at right angles (Sec. IV-D3).  By symmetry A's witness is the middle
    of its edge, (0.5, 0, 0.5), exactly; B's witness lies on its lowest edge (y = 0,
    z = 0.5 - delta), pulled along x only by the QP's alpha-space smoothing.  A's witness
    sits inside B, both soft signs are -1, so both signed distances are -|e1* - e2*|
    (<= -delta), the two normals are exactly opposite (n1 = -n2), n1 points down into A
    (B's outward side there), and the normals clash (cl ~ 1)."""
    from oracle.manifold import _Body
    import synth
    box = synth.primitive_geometry(synth.KIND_BOX)
    tau, delta = 1e-2, 0.05
    c, s = np.cos(np.pi / 8), np.sin(np.pi / 8)
    A = _Body(box, t([1, 0, 0, 0, 0, 0, 0]), t([0.5, 0.5, 0.5]), tau)
    B = _Body(box, t([c, s, 0, 0, 0, 0, 0.5 - delta + np.sqrt(0.5)]), t([1.0, 0.5, 0.5]), tau)
    a0, a1 = A.verts[A.edges[:, 0]], A.verts[A.edges[:, 1]]
    b0, b1 = B.verts[B.edges[:, 0]], B.verts[B.edges[:, 1]]
    cand = oracle.ee_candidates(a0, a1, b0, b1, A.sdf, B.sdf, tau)
    miss = (cand["p1"] - t([0.5, 0, 0.5])).norm(dim=-1)
    miss = miss + (cand["p2"][..., 1:] - t([0, 0.5 - delta])).norm(dim=-1)
    k, l = np.unravel_index(int(torch.argmin(miss)), miss.shape)
    p1, p2 = cand["p1"][k, l].numpy(), cand["p2"][k, l].numpy()
    np.testing.assert_allclose(p1, [0.5, 0, 0.5], atol=1e-12)
    np.testing.assert_allclose(p2[1:], [0, 0.5 - delta], atol=1e-12)
    assert abs(p2[0] - 0.5) < 2e-2
    g1, g2 = float(cand["gamma1"][k, l]), float(cand["gamma2"][k, l])
    assert g1 < -0.999999 and g2 < -0.999999
    dbar = np.linalg.norm(p1 - p2)
    assert dbar >= delta
    for d in (float(cand["d1"][k, l]), float(cand["d2"][k, l])):
        assert abs(d + dbar) < 1e-9, (d, dbar)
    n1, n2 = cand["n1"][k, l].numpy(), cand["n2"][k, l].numpy()
    np.testing.assert_allclose(n1, -n2, atol=1e-12)
    assert n1[2] < -0.9 and abs(n1[1]) < 1e-9
    assert float(cand["pen1"][k, l]) > 0.9
    assert float(cand["cl"][k, l]) > 0.99
    # nearest-neighbour indicators: A's edge has one near edge of B (nn over B's edges
    # ~ 1); B's lowest edge crosses both of A's top edges along y, at x = +-0.5, at
    # mirror-equal distances (nn over A's edges = 1/2; the next edges are ~0.45 farther)
    assert float(cand["nn1"][k, l]) > 0.999
    assert abs(float(cand["nn2"][k, l]) - 0.5) < 1e-9
