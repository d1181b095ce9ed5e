"""The kernels' superquadric-union SDF and its hand-written reverse, built for the
host, against the FP64 oracle.

A multi-primitive body (Sec. IV-B, IV-B1) is the smooth union phi = -LSE_tau(-phi_l)
of superquadrics phi_l = (1 - f_l^(-eps1/2)) |x| in each primitive's frame; its normal
blends the primitives' grad f with the union's weights.  The kernels evaluate every
power as an exp2 of base-2 logarithms; ``tests/host/sq_union_check.cu`` builds the
forward (``sdf_sq_union``) and its reverse through the normal (``normal_bwd``,
``sdf_sq_union_bwd``) for the CPU.  Here both are held to the oracle's ``sdf_local`` and
its autograd on random unions of 5 and 18 superquadrics (exponents 0.3 .. 1.5) at
tau 1e-2 and 1e-1, at mesh vertices (on the surface), near them and in the body's
bounding box.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import synth
from oracle.sdf import SQ_UNION, sdf_local

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "sq_union_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "sq_union_check")
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


@pytest.mark.parametrize("n_prims", [5, 18])
@pytest.mark.parametrize("tau", [1e-2, 1e-1])
def test_union_value_normal_and_reverse(exe, n_prims, tau):
    rng = np.random.default_rng(n_prims * 10 + int(round(-np.log10(tau))))
    g = synth.random_sq_union(rng, n_prims)
    rows = g.planes.reshape(n_prims, 12).astype(np.float64)
    v = g.verts[:, :3].astype(np.float64)
    lo, hi = v.min(0) - 0.1, v.max(0) + 0.1
    pick = rng.choice(len(v), 20, replace=False)
    y = np.concatenate([v[pick], v[pick[:20]] + rng.normal(size=(20, 3)) * 3 * tau,
                        rng.uniform(lo, hi, size=(20, 3))]).astype(np.float32).astype(np.float64)
    phibar, nubar = rng.normal(size=len(y)), rng.normal(size=(len(y), 3))
    lines = [f"{tau!r} {n_prims}"] + [" ".join(f"{x:.9g}" for x in r) for r in rows]
    lines += [" ".join(f"{x:.9g}" for x in np.r_[a, b, c]) for a, b, c in zip(y, phibar, nubar)]
    res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    got = np.array([[float(x) for x in ln.split()] for ln in res.stdout.strip().splitlines()])
    assert got.shape == (len(y), 7)
    planes = torch.tensor(g.planes, dtype=F64)
    worst = {"phi": 0.0, "nu": 0.0, "grad": 0.0}
    for i in range(len(y)):
        yt = torch.tensor(y[i], dtype=F64, requires_grad=True)
        phi, nu = sdf_local(SQ_UNION, yt, torch.ones(3, dtype=F64), planes, tau)
        loss = phibar[i] * phi + (torch.tensor(nubar[i], dtype=F64) * nu).sum()
        (yb,) = torch.autograd.grad(loss, yt)
        worst["phi"] = max(worst["phi"], abs(got[i, 0] - float(phi.detach())))
        worst["nu"] = max(worst["nu"], np.abs(got[i, 1:4] - nu.detach().numpy()).max())
        worst["grad"] = max(worst["grad"], np.abs(got[i, 4:7] - yb.numpy()).max() / np.abs(yb.numpy()).max())
    assert worst["phi"] <= 1e-5 and worst["nu"] <= 1e-4 and worst["grad"] <= 1e-3, worst
