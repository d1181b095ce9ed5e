"""Smooth stand-ins for non-smooth operators (Sec. III; Supplement C, smooth operators).

Test infrastructure (see ``oracle/__init__``).  All functions take float64
tensors.  Pins: tests/test_oracle_smooth.py (exact identities, bounds and the
hard-operator limits as the smoothing goes to zero).
"""
import torch


def softplus(x):
    """log(1 + e^x), evaluated without overflow as max(x, 0) + log1p(e^-|x|)."""
    return torch.clamp(x, min=0.0) + torch.log1p(torch.exp(-torch.abs(x)))


def sigmoid(x):
    """Logistic function 1 / (1 + e^-x) (Sec. III)."""
    return torch.sigmoid(x)


def relu_s(x, eps):
    """Smooth ReLU: eps * log(1 + exp(x / eps)) (Sec. III)."""
    return eps * softplus(x / eps)


def clip_s(x, lo, hi, eps):
    """Soft clip: lo + relu_s(x - lo) - relu_s(x - hi) (Sec. III)."""
    return lo + relu_s(x - lo, eps) - relu_s(x - hi, eps)


def greater_s(x, lo, eps):
    """Soft Iverson bracket [x > lo] = sigmoid((x - lo) / eps) (Sec. III)."""
    return torch.sigmoid((x - lo) / eps)


def smaller_s(x, hi, eps):
    """Soft Iverson bracket [x < hi] = sigmoid((hi - x) / eps) (Sec. III)."""
    return torch.sigmoid((hi - x) / eps)


def within_s(x, lo, hi, eps):
    """Soft indicator of lo <= x <= hi as the product of the two soft comparisons."""
    return greater_s(x, lo, eps) * smaller_s(x, hi, eps)


def argmin_s(x, eps, dim=-1):
    """Soft argmin: softmax(-x / eps) along ``dim`` (Sec. III, soft argmax of -x)."""
    return torch.softmax(-x / eps, dim=dim)


def lse(x, tau, dim=-1):
    """Real-softmax tau * log sum exp(x / tau) along ``dim`` (Sec. III)."""
    return tau * torch.logsumexp(x / tau, dim=dim)


def sign_s(x, eps):
    """Soft sign tanh(x / eps) (Sec. III)."""
    return torch.tanh(x / eps)
