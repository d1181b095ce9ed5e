"""The kernels' polyhedron SDF routines compiled for the host, against the closed form.

The smooth polyhedron SDF is a log-sum-exp over the face planes at softness tau
(Sec. IV-B2): phi(y) = tau ln sum_f exp((n_f . y - c_f) / tau), grad phi = sum_f pi_f n_f
with pi = softmax((n . y - c) / tau), and Hessian (sum_f pi_f n_f n_f^T - g g^T) / tau.
The adjoint evaluates it at an edge pair's two witnesses in one pass over the planes,
either with a running maximum (``sdf_planes2_h``) or, while the body's own witness y2 is
within a scaled distance of 60 of its edge, as plain sums (``sdf_planes2_h_ee``).  The
plain form lets the sum at the other body's witness y1 overflow or underflow; there the
penetration indicator sigma(-phi(y1) / tau) is exactly 0 or 1 and its derivative, the
only factor that multiplies grad phi(y1), is 0, so that gradient is returned as 0.

Here both routines run in FP32 on the CPU (``tests/host/hull_sdf_check.cu`` includes the
kernels' header; exp2 / log2 / division replace the MUFU instructions) and are held to
the FP64 closed form on random polytopes at tau in {1e-3, 1e-2, 1e-1}, and the plain
form's saturated cases are checked to give infinite values and zero gradients, never NaN.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "hull_sdf_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "hull_sdf_check")
LOG2E = 1.4426950408889634


@pytest.fixture(scope="module")
def exe():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is needed to build the host check")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    deps = [SRC, os.path.join(CSRC, "cm_math.cuh")]
    if not os.path.exists(EXE) or any(os.path.getmtime(d) > os.path.getmtime(EXE) for d in deps):
        subprocess.run([nvcc, "-std=c++17", "-O2", f"-I{CSRC}", SRC, "-o", EXE], check=True,
                       capture_output=True)
    return EXE


def run(exe, tau, planes, y1, y2):
    lines = [f"{tau!r} {len(planes)}"] + [" ".join(f"{v:.9g}" for v in row) for row in planes]
    lines += [" ".join(f"{v:.9g}" for v in np.r_[a, b]) for a, b in zip(y1, y2)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    rows = np.array([[float(v) for v in ln.split()] for ln in out.stdout.strip().splitlines()])
    assert rows.shape == (len(y1), 28)

    def unpack(r):
        return {"phi1": r[:, 0], "g1": r[:, 1:4], "phi2": r[:, 4], "g2": r[:, 5:8], "H": r[:, 8:14]}
    return unpack(rows[:, :14]), unpack(rows[:, 14:])


def closed_form(tau, planes, y):
    """FP64 log-sum-exp SDF, gradient and Hessian (xx, xy, xz, yy, yz, zz) at points y."""
    n, c = planes[:, :3].astype(np.float64), planes[:, 3].astype(np.float64)
    s = (y @ n.T - c) / tau
    m = s.max(axis=1, keepdims=True)
    e = np.exp(s - m)
    S = e.sum(axis=1, keepdims=True)
    pi = e / S
    phi = tau * (m[:, 0] + np.log(S[:, 0]))
    g = pi @ n
    nn = np.einsum("fi,fj->fij", n, n)
    H = (np.einsum("pf,fij->pij", pi, nn) - np.einsum("pi,pj->pij", g, g)) / tau
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    return phi, g, np.stack([H[:, i, j] for i, j in iu], axis=1)


def polytope(rng, F):
    n = rng.normal(size=(F, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return np.c_[n, rng.uniform(0.5, 1.0, F)].astype(np.float32).astype(np.float64)


def boundary_point(planes, d):
    """The point of the polytope's boundary along the unit direction d from the origin."""
    nd = planes[:, :3] @ d
    return d * np.min(planes[nd > 1e-9, 3] / nd[nd > 1e-9])


def sigma_neg(phi, tau):
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(np.clip(phi / tau, -700, 700)))


# FP32 evaluation of phi near unit scale is good to a few 1e-8 absolute (plane values of
# magnitude up to ~3 / tau rounded to 2^-24 relative, then scaled back by tau); the
# indicator sigma(-phi / tau) carries that error times its slope pen (1 - pen) / tau.
PHI_TOL = 5e-7


def check_indicator_and_gradient(form, phi1, g1, tau):
    pen = sigma_neg(phi1, tau)
    fin = np.isfinite(form["phi1"])
    assert (np.abs(form["phi1"][fin] - phi1[fin]) <= PHI_TOL * np.maximum(1.0, np.abs(phi1[fin]))).all()
    slope = pen * (1 - pen)
    assert (np.abs(sigma_neg(form["phi1"], tau) - pen) <= slope * (PHI_TOL / tau) + 1e-9).all()
    # grad phi(y1) only enters through the indicator's derivative, a multiple of the slope
    assert np.isfinite(form["g1"]).all()
    assert (slope * np.abs(form["g1"] - g1).max(axis=1)).max() <= 1e-6


@pytest.mark.parametrize("tau", [1e-3, 1e-2, 1e-1])
def test_both_forms_match_the_closed_form(exe, tau):
    rng = np.random.default_rng(int(round(-np.log10(tau))) + 40)
    for trial in range(12):
        planes = polytope(rng, int(rng.integers(8, 500)))
        d = rng.normal(size=(16, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        y2 = np.array([boundary_point(planes, v) for v in d])
        y2 += rng.normal(size=y2.shape) * (0.5 * tau)           # near the surface, either side
        y1 = np.where(np.arange(16)[:, None] % 2 == 0, y2 + rng.normal(size=y2.shape) * (5 * tau),
                      rng.uniform(-1.5, 1.5, size=y2.shape))
        y1, y2 = y1.astype(np.float32).astype(np.float64), y2.astype(np.float32).astype(np.float64)
        phi1, g1, _ = closed_form(tau, planes, y1)
        phi2, g2, H2 = closed_form(tau, planes, y2)
        for form in run(exe, tau, planes, y1, y2):
            assert np.isfinite(form["phi2"]).all() and np.isfinite(form["H"]).all()
            assert np.abs(form["phi2"] - phi2).max() <= PHI_TOL
            assert np.abs(form["g2"] - g2).max() <= 1e-5
            assert (np.abs(form["H"] - H2) * tau).max() <= 1e-4
            check_indicator_and_gradient(form, phi1, g1, tau)


def test_plain_sums_saturate_without_nan(exe):
    """At tau = 1e-3 the sum at y1 overflows far outside the body and underflows deep
    inside it; the plain form returns phi1 = +inf / -inf with a zero gradient there,
    and at every distance in between the dropped gradient is negligible."""
    tau = 1e-3
    rng = np.random.default_rng(7)
    planes = polytope(rng, 200)
    d = np.array([0.36, -0.48, 0.8])
    y2 = boundary_point(planes, d)
    k = LOG2E / tau
    steps = np.array([0.0, 20, 60, 100, 110, 120, 130, 200, 2000]) / k   # scaled distances
    y1 = np.vstack([y2 + s * d for s in steps] + [np.zeros(3), 0.2 * y2])
    y2s = np.repeat(y2[None], len(y1), axis=0)
    y1 = y1.astype(np.float32).astype(np.float64)
    shifted, plain = run(exe, tau, planes, y1, y2s)
    phi1, g1, _ = closed_form(tau, planes, y1)
    assert np.isfinite(plain["g1"]).all() and not np.isnan(plain["phi1"]).any()
    assert plain["phi1"][-4] == np.inf and not plain["g1"][-4].any()       # 2000 scaled units out
    assert plain["phi1"][-2] == -np.inf and not plain["g1"][-2].any()      # the centre
    assert np.isfinite(shifted["phi1"]).all()                              # the shifted form stays finite
    for form in (shifted, plain):
        check_indicator_and_gradient(form, phi1, g1, tau)
