"""The kernels' edge-edge box QP and its hand-written reverse, built for the host,
against the FP64 oracle.

The E-E witness routine (Sec. IV-D2) solves the regularised 2x2 box QP of two edges
with the smoothed analytic active set; the kernels evaluate it in FP32 with the
unconstrained solve in Lagrange / Binet-Cauchy form (one cross product carries the
near-parallel cancellation), and the adjoint reverses it by hand (``qp_bwd``).
``tests/host/qp_check.cu`` compiles both from the kernels' headers for the CPU (exp2 /
division in place of the MUFU instructions); here they are held to the oracle's
``ee_witness`` (FP64) and to its autograd vector-Jacobian product, on random edges,
edges 1e-6 .. 1e-2 rad from parallel, and edges whose unconstrained minimiser lies
outside the box.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from oracle.edge_edge import ee_witness

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "qp_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "qp_check")


@pytest.fixture(scope="module")
def exe():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is needed to build the host check")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    deps = [SRC] + [os.path.join(CSRC, f) for f in ("cm_math.cuh", "cm_adjoint.cuh")]
    if not os.path.exists(EXE) or any(os.path.getmtime(d) > os.path.getmtime(EXE) for d in deps):
        subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{CSRC}", SRC, "-o", EXE], check=True,
                       capture_output=True)
    return EXE


def run(exe, ends, bars):
    """ends (n, 4, 3) FP32-representable endpoints, bars (n, 3) -> (alpha, con) (n, 3) and
    endpoint adjoints (n, 4, 3)."""
    lines = [" ".join(f"{x:.9g}" for x in np.r_[e.ravel(), b]) for e, b in zip(ends, bars)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    rows = np.array([[float(x) for x in ln.split()] for ln in out.stdout.strip().splitlines()])
    assert rows.shape == (len(ends), 15)
    return rows[:, :3], rows[:, 3:].reshape(-1, 4, 3)


def oracle(ends, bars):
    x = torch.tensor(ends, dtype=torch.float64, requires_grad=True)
    _, _, a1, a2, con = ee_witness(x[:, 0], x[:, 1], x[:, 2], x[:, 3])
    out = torch.stack([a1, a2, con], dim=1)
    (g,) = torch.autograd.grad(out, x, torch.tensor(bars, dtype=torch.float64))
    return out.detach().numpy(), g.numpy()


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def near_parallel(rng, n):
    """Edge pairs whose directions are 1e-6 .. 1e-2 rad apart, overlapping along them."""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = rng.normal(size=(n, 3))
    p -= (p * d).sum(1, keepdims=True) * d
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    ang = 10.0 ** rng.uniform(-6, -2, n)
    d2 = np.cos(ang)[:, None] * d + np.sin(ang)[:, None] * p
    c = rng.uniform(-0.5, 0.5, size=(n, 3))
    off = rng.normal(size=(n, 3)) * 0.2
    L1, L2 = rng.uniform(0.3, 1.0, (2, n, 1))
    s = rng.uniform(-0.3, 0.3, (n, 1))
    return np.stack([c - L1 * d, c + L1 * d, c + off + (s - L2) * d2, c + off + (s + L2) * d2], axis=1)


def test_qp_values_match_the_oracle(exe):
    rng = np.random.default_rng(5)
    general = rng.uniform(-1, 1, size=(400, 4, 3))
    ends = f32(np.concatenate([general, near_parallel(rng, 400)]))
    bars = rng.normal(size=(len(ends), 3))
    got, _ = run(exe, ends, bars)
    want, _ = oracle(ends, bars)
    err = np.abs(got - want).max(axis=0)
    assert (err <= 1e-5).all(), err
    assert want[:, 2].min() < 0.05 and want[:, 2].max() > 0.95      # both regimes of con occur


def test_qp_reverse_matches_the_oracle_autograd(exe):
    """Endpoint adjoints of abar . (alpha1, alpha2, con) within 1e-3 of each case's largest
    component (the gradient bar), on general edges and on edges 1e-6 .. 1e-2 rad from
    parallel (measured: 6e-5 and 8e-5 at most)."""
    rng = np.random.default_rng(6)
    ends = f32(np.concatenate([rng.uniform(-1, 1, size=(400, 4, 3)), near_parallel(rng, 400)]))
    bars = rng.normal(size=(len(ends), 3))
    _, got = run(exe, ends, bars)
    _, want = oracle(ends, bars)
    scale = np.abs(want).reshape(len(ends), -1).max(axis=1)
    rel = np.abs(got - want).reshape(len(ends), -1).max(axis=1) / scale
    assert rel.max() <= 1e-3, (rel.max(), int(np.argmax(rel)))
