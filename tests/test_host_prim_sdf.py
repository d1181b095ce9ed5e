"""The kernels' smooth primitive SDFs and their hand-written reverses, built for the
host, against the FP64 oracle.

Box (LSE over six planes), capsule (soft-clipped axis), cylinder (LSE of the radial
and cap distances) and ellipsoid (the superquadric with eps1 = eps2 = 1), Sec. IV-B,
with the normal g / sqrt(tau + |g|^2) of Sec. IV-C.  ``tests/host/prim_sdf_check.cu``
compiles the kernels' forward (``prim_sdf``) and reverse (``normal_bwd`` then
``prim_sdf_bwd``) for the CPU; here the value and normal are held to the oracle's
``sdf_local`` (FP64) and the point and dims adjoints of phibar phi + nubar . nu to the
oracle's autograd, at tau in {1e-3, 1e-2, 1e-1}, on points inside, near and outside
each surface.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from oracle.sdf import sdf_local

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "prim_sdf_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "prim_sdf_check")
KINDS = {"box": 0, "capsule": 1, "cylinder": 2, "ellipsoid": 3}


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


def cases(rng, kind, n):
    dims = rng.uniform(0.2, 1.0, size=(n, 3))
    if kind in ("capsule", "cylinder"):
        dims[:, 2] = 0.0                                   # (radius, half-length, unused)
        ext = np.c_[dims[:, 0], dims[:, 0], dims[:, 1] + (dims[:, 0] if kind == "capsule" else 0)]
    else:
        ext = dims
    u = rng.uniform(-1.0, 1.0, size=(n, 3))
    scale = np.where(np.arange(n)[:, None] % 2 == 0, 1.0 + 0.02 * rng.normal(size=(n, 1)),
                     rng.uniform(0.3, 1.6, size=(n, 1)))   # half of them near the surface
    y = u / np.abs(u).max(axis=1, keepdims=True) * ext * scale
    return f32(y), f32(dims)


def run(exe, kind, tau, y, dims, phibar, nubar):
    lines = [f"{KINDS[kind]} {tau!r} " + " ".join(f"{x:.9g}" for x in np.r_[a, d, pb, nb])
             for a, d, pb, nb in zip(y, dims, phibar, nubar)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    r = np.array([[float(x) for x in ln.split()] for ln in out.stdout.strip().splitlines()])
    assert r.shape == (len(y), 10)
    return r[:, 0], r[:, 1:4], r[:, 4:7], r[:, 7:10]


def oracle(kind, tau, y, dims, phibar, nubar):
    phis, nus, ybs, dbs = [], [], [], []
    for i in range(len(y)):
        yt = torch.tensor(y[i], dtype=torch.float64, requires_grad=True)
        dt = torch.tensor(dims[i], dtype=torch.float64, requires_grad=True)
        d_used = dt if kind in ("box", "ellipsoid") else dt[:2]
        phi, nu = sdf_local(KINDS[kind], yt, d_used, None, tau)
        loss = phibar[i] * phi + (torch.tensor(nubar[i], dtype=torch.float64) * nu).sum()
        yb, db = torch.autograd.grad(loss, (yt, dt), allow_unused=True)
        phis.append(float(phi.detach()))
        nus.append(nu.detach().numpy())
        ybs.append(yb.numpy())
        dbs.append(np.zeros(3) if db is None else db.numpy())
    return np.array(phis), np.array(nus), np.array(ybs), np.array(dbs)


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("tau", [1e-3, 1e-2, 1e-1])
def test_primitive_value_normal_and_reverse(exe, kind, tau):
    rng = np.random.default_rng(100 * KINDS[kind] + int(round(-np.log10(tau))))
    y, dims = cases(rng, kind, 60)
    phibar, nubar = rng.normal(size=60), rng.normal(size=(60, 3))
    phi, nu, yb, db = run(exe, kind, tau, y, dims, phibar, nubar)
    phi_o, nu_o, yb_o, db_o = oracle(kind, tau, y, dims, phibar, nubar)
    assert np.abs(phi - phi_o).max() <= 1e-5
    assert np.abs(nu - nu_o).max() <= 1e-4
    g, g_o = np.c_[yb, db], np.c_[yb_o, db_o]
    rel = np.abs(g - g_o).max(axis=1) / np.abs(g_o).max(axis=1)
    assert rel.max() <= 1e-3, (rel.max(), int(np.argmax(rel)))
