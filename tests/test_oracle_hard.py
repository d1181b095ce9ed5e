"""Pins of the oracle's non-smoothed witness routines (the paper's Ours-NS, Sec. V) against
optimality conditions and brute force.

E-E: the regularised box QP is strictly convex, so its minimiser over [0, 1]^2 is unique
and certified by the KKT conditions: with g = Q alpha + c, each coordinate has g_i = 0
where 0 < alpha_i < 1, g_i >= 0 at alpha_i = 0 and g_i <= 0 at alpha_i = 1.
V-F: p is the closest point of a triangle to v exactly when (v - p) . (T_i - p) <= 0 for
the three corners (a convex set's projection condition, checked on its extreme points).
"""
import numpy as np
import pytest
import torch

from oracle.edge_edge import ee_witness, solve_box_qp, solve_box_qp_hard
from oracle.vertex_face import vf_witness

F = torch.float64


def t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), dtype=F)


def qp_terms(a0, a1, b0, b1, lam):
    t1, t2, b = a1 - a0, b0 - b1, a0 - b0
    return (t1 @ t1 + lam, t1 @ t2, t2 @ t2 + lam, t1 @ b - 0.5 * lam, t2 @ b - 0.5 * lam)


@pytest.mark.parametrize("seed", range(40))
def test_ee_hard_satisfies_kkt(seed):
    rng = np.random.default_rng(300 + seed)
    a0, a1, b0, b1 = rng.uniform(-1, 1, size=(4, 3))
    lam = 0.01
    _, _, al1, al2, con = ee_witness(t(a0), t(a1), t(b0), t(b1), w_reg=lam, hard=True)
    Q11, Q12, Q22, c1, c2 = qp_terms(a0, a1, b0, b1, lam)
    al = np.array([al1.item(), al2.item()])
    g = np.array([Q11 * al[0] + Q12 * al[1] + c1, Q12 * al[0] + Q22 * al[1] + c2])
    for i in range(2):
        assert -1e-15 <= al[i] <= 1 + 1e-15
        if al[i] <= 0.0:
            assert g[i] >= -1e-12
        elif al[i] >= 1.0:
            assert g[i] <= 1e-12
        else:
            assert abs(g[i]) < 1e-12
    assert con.item() in (0.0, 1.0)


@pytest.mark.parametrize("seed", range(8))
def test_ee_hard_matches_dense_grid(seed):
    rng = np.random.default_rng(400 + seed)
    a0, a1, b0, b1 = rng.uniform(0, 1, size=(4, 3))
    lam = 0.01
    gr = np.linspace(0, 1, 1001)
    A1, A2 = np.meshgrid(gr, gr, indexing="ij")
    e1 = a0 + A1[..., None] * (a1 - a0)
    e2 = b0 + A2[..., None] * (b1 - b0)
    J = ((e1 - e2) ** 2).sum(-1) + lam * ((A1 - 0.5) ** 2 + (A2 - 0.5) ** 2)
    i = np.unravel_index(np.argmin(J), J.shape)
    _, _, al1, al2, _ = ee_witness(t(a0), t(a1), t(b0), t(b1), w_reg=lam, hard=True)
    assert abs(al1.item() - gr[i[0]]) < 2e-3 and abs(al2.item() - gr[i[1]]) < 2e-3


def test_ee_hard_is_the_smooth_solve_in_the_limit():
    rng = np.random.default_rng(7)
    for _ in range(50):
        Q11, Q12, Q22, c1, c2 = qp_terms(*rng.uniform(-1, 1, size=(4, 3)), 0.01)
        args = [t(x) for x in (Q11, Q12, Q22, c1, c2)]
        h = solve_box_qp_hard(*args)
        s = solve_box_qp(*args, eps_clip=1e-9, eps_min=1e-9, eps_comp=1e-9)
        assert abs(h[0].item() - s[0].item()) < 1e-6 and abs(h[1].item() - s[1].item()) < 1e-6


def test_ee_hard_interior_and_corner_cases():
    # skew perpendicular edges crossing at their midpoints h apart: interior, con = 1
    _, _, al1, al2, con = ee_witness(t([-1, 0, 0]), t([1, 0, 0]), t([0, -1, 0.5]), t([0, 1, 0.5]), hard=True)
    assert abs(al1.item() - 0.5) < 1e-14 and abs(al2.item() - 0.5) < 1e-14 and con.item() == 1.0
    # edges that meet end to end far from each other's interior: a corner, con = 0
    _, _, al1, al2, con = ee_witness(t([0, 0, 0]), t([1, 0, 0]), t([2, 0, 1]), t([3, 0, 2]), hard=True)
    assert al1.item() == 1.0 and al2.item() == 0.0 and con.item() == 0.0


def tri(rng):
    while True:
        T = rng.uniform(-1, 1, size=(3, 3))
        if np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0])) > 0.3:
            return T


@pytest.mark.parametrize("seed", range(40))
def test_vf_hard_is_the_projection(seed):
    rng = np.random.default_rng(500 + seed)
    T = tri(rng)
    v = rng.uniform(-1.5, 1.5, 3)
    p, inside = vf_witness(t(v), t(T[0]), t(T[1]), t(T[2]), hard=True)
    p = p.numpy()
    for c in T:
        assert (v - p) @ (c - p) <= 1e-12
    n = np.cross(T[1] - T[0], T[2] - T[0])
    assert abs((p - T[0]) @ n) < 1e-12 * np.linalg.norm(n)      # p lies in the triangle's plane
    assert inside.item() in (0.0, 1.0)


@pytest.mark.parametrize("seed", range(6))
def test_vf_hard_matches_dense_sampling(seed):
    rng = np.random.default_rng(600 + seed)
    T = tri(rng)
    v = rng.uniform(-1.5, 1.5, 3)
    g = np.linspace(0, 1, 801)
    a, b = np.meshgrid(g, g, indexing="ij")
    m = a + b <= 1
    P = T[0] + a[m][:, None] * (T[1] - T[0]) + b[m][:, None] * (T[2] - T[0])
    ref = P[np.argmin(((P - v) ** 2).sum(1))]
    p, _ = vf_witness(t(v), t(T[0]), t(T[1]), t(T[2]), hard=True)
    assert np.linalg.norm(p.numpy() - v) <= np.linalg.norm(ref - v) + 1e-12
    assert np.abs(p.numpy() - ref).max() < 5e-3
