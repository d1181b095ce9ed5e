"""The adjoint's vertex-SDF element, built for the host, against the FP64 oracle.

A vertex candidate (Sec. IV-C) is a vertex of one body with the other body's smooth
signed distance, normal and activity sigma(-d / tau) at it.  ``vs_bwd`` reverses it by
hand: the SDF's reverse (a polyhedron's through its Hessian, a primitive's through its
closed form), the normal's, the vertex map to the dims and the relative pose, which
``pose_epilogue`` chains to the quaternion and translation.
``tests/host/vs_element_check.cu`` builds them for the CPU on the kernels'
hull-vs-primitive pair class (A a convex polyhedron, B a box at the origin); here the
gradient with respect to A's quaternion and translation and B's half-extents is held
to the oracle's autograd of the same vertex rows (``pair_candidates``), for vertices
of both bodies of placed pairs at tau 1e-3, 1e-2 and 1e-1.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import synth
from oracle.manifold import _Body
from test_host_ee_element import box_pairs, f32

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "vs_element_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "vs_element_check")
F64 = torch.float64


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


def oracle_vertex(ga, gb, side, vi, qA, tA, hB, tau, ybar):
    x = torch.tensor(np.r_[qA, tA, hB], dtype=F64, requires_grad=True)
    A = _Body(ga, x[:7], torch.ones(3, dtype=F64), tau)
    B = _Body(gb, torch.tensor([1.0, 0, 0, 0, 0, 0, 0], dtype=F64), x[7:], tau)
    own, other = (A, B) if side == 0 else (B, A)
    v = own.verts[vi][None]
    phi, nu = other.sdf(v)
    w = torch.sigmoid(-phi / tau)
    row = torch.cat([v[0], phi, nu[0], w, -(w * phi)])
    (grad,) = torch.autograd.grad((row * torch.tensor(ybar, dtype=F64)).sum(), x)
    return grad.numpy()


@pytest.mark.parametrize("tau", [1e-3, 1e-2, 1e-1])
def test_vertex_element_matches_the_oracle(exe, tau):
    rng = np.random.default_rng(int(round(-np.log10(tau))) + 90)
    worst = 0.0
    for ga, gb, qA, tA, hB in box_pairs(tau, 4, seed=synth.SEED_BASE + 32):
        pl = f32(ga.planes)
        lines = [f"{tau!r} {len(pl)}"] + [" ".join(f"{v:.9g}" for v in r) for r in pl]
        cases = []
        for side, n in ((0, ga.n_verts), (1, gb.n_verts)):
            for vi in rng.choice(n, min(n, 6), replace=False):
                v = ga.verts[vi, :3] if side == 0 else gb.verts[vi, :3]
                ybar = rng.normal(size=9)
                cases.append((side, vi, ybar))
                lines.append(f"{side} " + " ".join(f"{x:.9g}" for x in f32(np.r_[qA, tA, v, hB, ybar])))
        res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        got = np.array([[float(x) for x in ln.split()] for ln in res.stdout.strip().splitlines()])
        assert got.shape == (len(cases), 10)
        for (side, vi, ybar), g in zip(cases, got):
            want = oracle_vertex(ga, gb, side, vi, qA, tA, hB, tau, ybar)
            worst = max(worst, np.abs(g - want).max() / np.abs(want).max())
    assert worst <= 1e-3, worst
