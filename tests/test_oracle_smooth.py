"""Pins of the oracle's smooth operators (Sec. III) against exact identities and hard limits."""
import numpy as np
import pytest
import torch

import oracle

F = torch.float64


def t(x):
    return torch.as_tensor(x, dtype=F)


@pytest.mark.parametrize("eps", [1e-3, 1e-2, 0.1, 1.0])
def test_clip_s_midpoint_exact(eps):
    # softplus(x) - softplus(-x) = x, so the soft clip of the midpoint is the midpoint.
    assert abs(oracle.clip_s(t(0.5), 0.0, 1.0, eps).item() - 0.5) < 1e-14


def test_softplus_identity_and_stability():
    x = t(np.linspace(-800, 800, 4001))
    sp = oracle.softplus(x)
    assert torch.isfinite(sp).all()
    assert torch.allclose(sp - oracle.softplus(-x), x, rtol=0, atol=1e-12)
    # against log1p(exp(x)) where that is representable
    xs = t(np.linspace(-30, 30, 601))
    assert torch.allclose(oracle.softplus(xs), torch.log1p(torch.exp(xs)), rtol=1e-14, atol=1e-300)


def test_relu_s_limit():
    x = t(np.linspace(-2, 2, 401))
    for eps in (1e-2, 1e-3, 1e-4):
        err = (oracle.relu_s(x, eps) - torch.clamp(x, min=0)).abs().max().item()
        assert err <= eps * np.log(2) + 1e-15


def test_clip_s_limit_and_range():
    x = t(np.linspace(-3, 3, 601))
    for eps in (1e-2, 1e-3):
        y = oracle.clip_s(x, -1.0, 2.0, eps)
        assert (y - torch.clamp(x, -1.0, 2.0)).abs().max().item() <= 2 * eps * np.log(2) + 1e-12
        assert (y >= -1.0 - 1e-12).all() and (y <= 2.0 + 1e-12).all()


def test_comparisons_and_within():
    x = t(np.array([-1.0, -0.2, 0.3, 0.7, 1.2, 2.0]))
    hard_gt = (x > 0).to(F)
    assert torch.allclose(oracle.greater_s(x, 0.0, 1e-4), hard_gt, atol=1e-12)
    assert torch.allclose(oracle.smaller_s(x, 1.0, 1e-4), (x < 1.0).to(F), atol=1e-12)
    within = ((x >= 0) & (x <= 1)).to(F)
    assert torch.allclose(oracle.within_s(x, 0.0, 1.0, 1e-4), within, atol=1e-12)
    # sigmoid symmetry and the soft comparison at the threshold itself
    assert abs(oracle.greater_s(t(0.3), 0.3, 0.1).item() - 0.5) < 1e-15
    assert torch.allclose(oracle.sigmoid(x) + oracle.sigmoid(-x), torch.ones_like(x), atol=1e-15)


def test_argmin_s_probabilities_and_limit():
    x = t(np.array([0.3, -0.1, 0.7, -0.05]))
    p = oracle.argmin_s(x, 0.1)
    assert abs(p.sum().item() - 1.0) < 1e-15 and (p > 0).all()
    assert int(torch.argmax(p)) == 1
    ph = oracle.argmin_s(x, 1e-4)
    assert torch.allclose(ph, torch.tensor([0, 1.0, 0, 0], dtype=F), atol=1e-12)
    pe = oracle.argmin_s(t([0.2, 0.2, 0.2]), 0.05)
    assert torch.allclose(pe, torch.full((3,), 1 / 3, dtype=F), atol=1e-15)


def test_lse_bounds():
    rng = np.random.default_rng(0)
    for tau in (1e-3, 1e-2, 1e-1):
        x = t(rng.normal(size=(50, 17)))
        v = oracle.lse(x, tau, dim=-1)
        mx = x.max(-1).values
        assert (v >= mx - 1e-14).all()
        assert (v <= mx + tau * np.log(17) + 1e-14).all()
    # N equal entries: exactly max + tau ln N
    assert abs(oracle.lse(t([0.4] * 6), 0.01).item() - (0.4 + 0.01 * np.log(6))) < 1e-15


def test_sign_s_limit():
    x = t(np.array([-0.5, -0.01, 0.02, 0.3]))
    assert torch.allclose(oracle.sign_s(x, 1e-5), torch.sign(x), atol=1e-12)
    assert oracle.sign_s(t(0.0), 0.1).item() == 0.0
