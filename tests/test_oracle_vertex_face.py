"""Pins of the oracle's vertex-face witness routine (Sec. IV-D1) against geometry."""
import numpy as np
import pytest
import torch

from oracle.vertex_face import vf_witness

F = torch.float64
HARD = dict(eps_clip=1e-8, eps_min=1e-8, eps_comp=1e-8)


def t(x):
    return torch.as_tensor(np.asarray(x), dtype=F)


def tri(rng):
    while True:
        T = rng.uniform(-1, 1, size=(3, 3))
        if np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0])) > 0.3:
            return T


def closest_brute(v, T, n=801):
    g = np.linspace(0, 1, n)
    a, b = np.meshgrid(g, g, indexing="ij")
    m = a + b <= 1
    P = T[0] + a[m][:, None] * (T[1] - T[0]) + b[m][:, None] * (T[2] - T[0])
    return P[np.argmin(((P - v) ** 2).sum(1))]


@pytest.mark.parametrize("seed", range(6))
def test_interior_projection_is_the_perpendicular_foot(seed):
    rng = np.random.default_rng(seed)
    T = tri(rng)
    w = rng.dirichlet([4, 4, 4])
    foot = w @ T
    n = np.cross(T[1] - T[0], T[2] - T[0])
    v = foot + rng.uniform(0.1, 1.0) * n / np.linalg.norm(n)
    got, inside = vf_witness(t(v), t(T[0]), t(T[1]), t(T[2]), **HARD)
    assert np.abs(got.numpy() - foot).max() < 1e-9 and abs(inside.item() - 1) < 1e-9


@pytest.mark.parametrize("seed", range(10))
def test_hard_limit_matches_brute_force(seed):
    rng = np.random.default_rng(50 + seed)
    T = tri(rng)
    v = rng.uniform(-1.5, 1.5, 3)
    got, _ = vf_witness(t(v), t(T[0]), t(T[1]), t(T[2]), **HARD)
    ref = closest_brute(v, T)
    assert np.linalg.norm(got.numpy() - v) <= np.linalg.norm(ref - v) + 1e-9
    assert np.abs(got.numpy() - ref).max() < 5e-3


@pytest.mark.parametrize("seed", range(6))
def test_relabelling_the_corners(seed):
    rng = np.random.default_rng(90 + seed)
    T = tri(rng)
    v = rng.uniform(-1.5, 1.5, 3)
    a, ia = vf_witness(t(v), t(T[0]), t(T[1]), t(T[2]))
    b, ib = vf_witness(t(v), t(T[1]), t(T[2]), t(T[0]))
    c, ic = vf_witness(t(v), t(T[2]), t(T[0]), t(T[1]))
    assert torch.allclose(a, b, atol=1e-13) and torch.allclose(a, c, atol=1e-13)
    assert abs(ia.item() - ib.item()) < 1e-13


def test_vertex_at_a_corner_and_on_an_edge():
    T = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    got, _ = vf_witness(t([1.5, -0.3, 0.7]), t(T[0]), t(T[1]), t(T[2]), **HARD)
    assert np.abs(got.numpy() - [1, 0, 0]).max() < 1e-7          # closest to corner T1
    got, _ = vf_witness(t([0.4, -0.5, 0.2]), t(T[0]), t(T[1]), t(T[2]), **HARD)
    assert np.abs(got.numpy() - [0.4, 0, 0]).max() < 1e-7        # closest to edge T0-T1
