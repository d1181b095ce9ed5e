"""The kernels' sphere tracing of E-E witnesses and its hand-written reverse, built for
the host, against the FP64 oracle.

Sphere tracing (Supplement, mesh-SDF discrepancies) moves a witness onto its own
body's smooth SDF surface by ``iters`` steps x <- x - phi(x) u along the fixed
direction u = grad phi(x0) / |grad phi(x0)|.  ``tests/host/trace_check.cu`` builds the
kernels' forward (``trace_to_surface``) and reverse (``trace_bwd``, which runs the
steps backwards and hands the direction's adjoint to the SDF gradient's adjoint at x0)
for the CPU.  Here the traced point and the adjoints of xbar . x_traced with respect to
the start point and the primitive's dims are held to the oracle's ``trace_to_surface``
and its autograd, for every primitive kind and a convex polyhedron, with 1 to 3 steps,
from points near the surface.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import synth
from oracle.edge_edge import trace_to_surface
from oracle.sdf import sdf_local

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "trace_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "trace_check")
F64 = torch.float64
KINDS = {"box": 0, "capsule": 1, "cylinder": 2, "ellipsoid": 3, "hull": 4}


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


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("iters", [1, 3])
def test_trace_and_its_reverse(exe, kind, iters):
    tau = 1e-2
    rng = np.random.default_rng(KINDS[kind] * 10 + iters)
    n = 24
    dims = rng.uniform(0.3, 1.0, size=(n, 3))
    planes = np.zeros((0, 4))
    if kind in ("capsule", "cylinder"):
        dims[:, 2] = 0.0
    if kind == "hull":
        g = synth.hull_from_points(rng.normal(size=(40, 3)) / 1.5)
        planes = f32(g.planes)
        dims[:] = 1.0
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    x0 = u * rng.uniform(0.3, 0.9, size=(n, 1))              # inside or near the surface
    x0, dims = f32(x0), f32(dims)
    xbar = rng.normal(size=(n, 3))
    lines = [f"{KINDS[kind]} {tau!r} {iters} {len(planes)}"] + [" ".join(f"{v:.9g}" for v in r) for r in planes]
    lines += [" ".join(f"{v:.9g}" for v in np.r_[a, d, b]) for a, d, b in zip(x0, dims, xbar)]
    res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    got = np.array([[float(v) for v in ln.split()] for ln in res.stdout.strip().splitlines()])
    assert got.shape == (n, 9)
    pl = torch.tensor(planes, dtype=F64)
    worst_x, worst_g = 0.0, 0.0
    for i in range(n):
        xt = torch.tensor(x0[i], dtype=F64, requires_grad=True)
        dt = torch.tensor(dims[i], dtype=F64, requires_grad=True)
        d_used = dt[:2] if kind in ("capsule", "cylinder") else dt
        x = trace_to_surface(xt, lambda y: sdf_local(KINDS[kind], y, d_used, pl, tau), iters)  # noqa: B023
        xb, db = torch.autograd.grad((x * torch.tensor(xbar[i], dtype=F64)).sum(), (xt, dt), allow_unused=True)
        db = torch.zeros(3, dtype=F64) if db is None or kind == "hull" else db
        want = np.r_[xb.numpy(), db.numpy()]
        worst_x = max(worst_x, np.abs(got[i, :3] - x.detach().numpy()).max())
        worst_g = max(worst_g, np.abs(got[i, 3:] - want).max() / np.abs(want).max())
    assert worst_x <= 1e-5 and worst_g <= 1e-3, (worst_x, worst_g)
