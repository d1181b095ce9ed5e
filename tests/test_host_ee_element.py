"""The adjoint's E-E element, built for the host, against the FP64 oracle.

For one edge of a convex polyhedron A and one edge of a box B (the kernels'
hull-vs-primitive pair class; also the other way round) the element recomputes both witnesses' candidates
(Sec. IV-D3: QP witnesses, signed distances and normals through the soft sign, the
penetration and clashing indicators, the weights) and reverses them, the QP and the
pose chain by hand (``ee_bwd``, ``ee_qp_bwd``, ``pose_epilogue``).  With one edge per
body both nearest-neighbour indicators are 1, which the element sees through row and
column minima equal to the edge pair's own distance.  ``tests/host/ee_element_check.cu``
builds it for the CPU; here its candidates are held to the oracle's ``ee_candidates``
and its gradient with respect to A's quaternion and translation and B's half-extents
to the oracle's autograd, on edge pairs of placed hull-vs-box pairs at tau 1e-2 and
1e-1, where every element takes the polyhedron's plain (unshifted) sums.  The shifted
sums are taken only where the QP witness overshoots its own edge by more than a
scaled distance of 60 (about 0.04 units at tau = 1e-3), which needs an edge longer than
the unit-ball hulls have: a 3.2-long edge at tau = 1e-3 checks both kinds.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import synth
from oracle.edge_edge import ee_candidates
from oracle.manifold import _Body

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host", "ee_element_check.cu")
CSRC = os.path.join(ROOT, "paper_2602_20304_gb300", "csrc")
EXE = os.path.join(ROOT, "_build", "ee_element_check")
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


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def rot(q):
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def relative_to_b(p):
    """A's pose (q, t) in B's frame from a pair's world poses (14,)."""
    qB = p[7:11] / np.linalg.norm(p[7:11])
    qA = quat_mul(qB * np.array([1, -1, -1, -1]), p[0:4] / np.linalg.norm(p[0:4]))
    return f32(qA), f32(rot(qB).T @ (p[4:7] - p[11:14]))


def box_pairs(tau, n_pairs, seed):
    """Placed hull-vs-box pairs, re-expressed with B at the origin: (hull, box geometry,
    qA, tA, hB) with every number FP32-representable."""
    w = synth.config_hull_vs_primitive(n=4 * n_pairs, seed=seed, taus=(tau,))
    out = []
    for i in range(w.n_pairs):
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
        if gb.kind != synth.KIND_BOX:
            continue
        qA, tA = relative_to_b(w.poses[i].astype(np.float64))
        out.append((ga, gb, qA, tA, f32(w.dims[i, 3:])))
        if len(out) == n_pairs:
            break
    return out


def run_hull(exe, hull, tau, rows, cls=1):
    pl = f32(hull.planes)
    lines = [f"{tau!r} {len(pl)} {cls}"] + [" ".join(f"{v:.9g}" for v in r) for r in pl]
    lines += [" ".join(f"{v:.9g}" for v in f32(r)) for r in rows]
    res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    out = np.array([[float(v) for v in ln.split()] for ln in res.stdout.strip().splitlines()])
    assert out.shape == (len(rows), 29)
    return out


def element_errors(got_vals, want_vals, got_grad, want_grad):
    e = {"p": 0.0, "d": 0.0, "n": 0.0, "w": 0.0}
    for j in (0, 9):
        e["p"] = max(e["p"], np.abs(got_vals[j:j + 3] - want_vals[j:j + 3]).max())
        e["d"] = max(e["d"], abs(got_vals[j + 3] - want_vals[j + 3]))
        e["n"] = max(e["n"], np.abs(got_vals[j + 4:j + 7] - want_vals[j + 4:j + 7]).max())
        e["w"] = max(e["w"], abs(got_vals[j + 7] - want_vals[j + 7]))
    e["grad"] = np.abs(got_grad - want_grad).max() / np.abs(want_grad).max()
    return e


def within_bar(e):
    return e["p"] <= 1e-5 and e["d"] <= 1e-5 and e["n"] <= 1e-4 and e["w"] <= 1e-4 and e["grad"] <= 1e-3


def oracle_element(ga, gb, ea, eb, qA, tA, h, tau, ybar, cls=1):
    """Rows and gradient (qA, tA, h) of the oracle's element; h are the half-extents of
    the box, B in class 1 and A in class 2."""
    x = torch.tensor(np.r_[qA, tA, h], dtype=F64, requires_grad=True)
    one = torch.ones(3, dtype=F64)
    A = _Body(ga, x[:7], one if cls == 1 else x[7:], tau)
    B = _Body(gb, torch.tensor([1.0, 0, 0, 0, 0, 0, 0], dtype=F64), x[7:] if cls == 1 else one, tau)
    a0, a1 = A.verts[A.edges[ea, 0]][None], A.verts[A.edges[ea, 1]][None]
    b0, b1 = B.verts[B.edges[eb, 0]][None], B.verts[B.edges[eb, 1]][None]
    c = ee_candidates(a0, a1, b0, b1, A.sdf, B.sdf, tau)
    rows = []
    for j in (1, 2):
        y = torch.cat([c[f"p{j}"][0, 0], c[f"d{j}"][0, 0, None], c[f"n{j}"][0, 0], c[f"w{j}"][0, 0, None]])
        rows.append(torch.cat([y, -(y[7] * y[3])[None]]))
    vals = torch.cat(rows)
    (grad,) = torch.autograd.grad((vals * torch.tensor(ybar, dtype=F64)).sum(), x)
    return vals.detach().numpy(), grad.numpy()


@pytest.mark.parametrize("tau", [1e-2, 1e-1])
def test_element_matches_the_oracle(exe, tau):
    rng = np.random.default_rng(int(round(-np.log10(tau))) + 70)
    cases, meta = [], []
    for ga, gb, qA, tA, hB in box_pairs(tau, 6, seed=synth.SEED_BASE + 31):
        R = rot(qA)
        va = ga.verts[:, :3].astype(np.float64) @ R.T + tA
        vb = gb.verts[:, :3].astype(np.float64) * hB
        # the closest edge pairs by hard segment distance, then random ones
        d = np.array([[np.linalg.norm(0.5 * (va[a0] + va[a1]) - 0.5 * (vb[b0] + vb[b1]))
                       for b0, b1 in gb.edges] for a0, a1 in ga.edges])
        order = np.argsort(d, axis=None)
        picks = list(order[:4]) + list(rng.choice(d.size, 4, replace=False))
        for flat in picks:
            ea, eb = np.unravel_index(flat, d.shape)
            ybar = rng.normal(size=18)
            row = np.r_[qA, tA, ga.verts[ga.edges[ea, 0], :3], ga.verts[ga.edges[ea, 1], :3],
                        gb.verts[gb.edges[eb, 0], :3], gb.verts[gb.edges[eb, 1], :3], hB, ybar]
            cases.append(row)
            meta.append((ga, gb, ea, eb, qA, tA, hB, ybar))
    by_hull = {}
    for i, m in enumerate(meta):
        by_hull.setdefault(id(m[0]), []).append(i)
    plain_seen = 0
    for idx in by_hull.values():
        out = run_hull(exe, meta[idx[0]][0], tau, [cases[i] for i in idx])
        for i, row in zip(idx, out):
            ga, gb, ea, eb, qA, tA, hB, ybar = meta[i]
            plain_seen += int(row[28])
            want_vals, want_grad = oracle_element(ga, gb, ea, eb, qA, tA, hB, tau, ybar)
            e = element_errors(row[:18], want_vals, row[18:28], want_grad)
            assert within_bar(e), (i, e)
    assert plain_seen == len(meta)


def test_long_edge_takes_both_sums(exe):
    """A 3.2-long edge of a slab-shaped polyhedron against a box edge beyond its end, at
    tau = 1e-3: as the offset grows the soft-blended QP witness overshoots the edge's end
    by more than a scaled distance of 60, then less again; both kinds of sums are taken
    and each element meets the bar."""
    tau, half = 1e-3, 1.6
    ga = synth.hull_from_points(np.array([[x, y, z] for x in (-half, half) for y in (-0.2, 0.2)
                                          for z in (-0.2, 0.2)]))
    gb = synth.primitive_geometry(synth.KIND_BOX)
    hB = f32([0.3, 0.3, 0.3])
    va, vb = ga.verts[:, :3], gb.verts[:, :3] * hB
    on = lambda v, **c: all(abs(v[{"x": 0, "y": 1, "z": 2}[k]] - x) < 1e-6 for k, x in c.items())  # noqa: E731
    ea = next(i for i, (a, b) in enumerate(ga.edges) if on(va[a], y=0.2, z=0.2) and on(va[b], y=0.2, z=0.2))
    eb = next(i for i, (a, b) in enumerate(gb.edges) if on(vb[a], x=0.3, z=0.3) and on(vb[b], x=0.3, z=0.3))
    rng = np.random.default_rng(3)
    qA = np.array([1.0, 0.0, 0.0, 0.0])
    rows, meta = [], []
    for over in np.linspace(0.0, 0.8, 17):
        tA = f32([0.3 - over - half, 0.0, 0.09])
        ybar = rng.normal(size=18)
        rows.append(np.r_[qA, tA, ga.verts[ga.edges[ea, 0], :3], ga.verts[ga.edges[ea, 1], :3],
                          gb.verts[gb.edges[eb, 0], :3], gb.verts[gb.edges[eb, 1], :3], hB, ybar])
        meta.append((tA, ybar))
    out = run_hull(exe, ga, tau, rows)
    assert 0 < int(out[:, 28].sum()) < len(rows)
    for row, (tA, ybar) in zip(out, meta):
        want_vals, want_grad = oracle_element(ga, gb, ea, eb, qA, tA, hB, tau, ybar)
        e = element_errors(row[:18], want_vals, row[18:28], want_grad)
        assert within_bar(e), e


@pytest.mark.parametrize("tau", [1e-2, 1e-1])
def test_box_against_hull_element_matches_the_oracle(exe, tau):
    """The other specialised pair class: A a box, B the hull of 32 points on the unit
    sphere (the box-vs-hull differentiation setting), with B's polyhedron taking the
    plain sums; the dims gradient is the box's (A's)."""
    rng = np.random.default_rng(int(round(-np.log10(tau))) + 80)
    w = synth.config_box_vs_sphere_hull(n=4, seed=synth.SEED_BASE + 33, tau=tau)
    plain_seen, n_el = 0, 0
    for i in range(w.n_pairs):
        ga, gb = w.geoms[w.pair_geoms[i, 0]], w.geoms[w.pair_geoms[i, 1]]
        qA, tA = relative_to_b(w.poses[i].astype(np.float64))
        hA = f32(w.dims[i, :3])
        va = ga.verts[:, :3].astype(np.float64) * hA @ rot(qA).T + tA
        vb = gb.verts[:, :3].astype(np.float64)
        d = np.array([[np.linalg.norm(0.5 * (va[a0] + va[a1]) - 0.5 * (vb[b0] + vb[b1]))
                       for b0, b1 in gb.edges] for a0, a1 in ga.edges])
        picks = list(np.argsort(d, axis=None)[:4]) + list(rng.choice(d.size, 4, replace=False))
        rows, meta = [], []
        for flat in picks:
            ea, eb = np.unravel_index(flat, d.shape)
            ybar = rng.normal(size=18)
            rows.append(np.r_[qA, tA, ga.verts[ga.edges[ea, 0], :3], ga.verts[ga.edges[ea, 1], :3],
                              gb.verts[gb.edges[eb, 0], :3], gb.verts[gb.edges[eb, 1], :3], hA, ybar])
            meta.append((ea, eb, ybar))
        out = run_hull(exe, gb, tau, rows, cls=2)
        for row, (ea, eb, ybar) in zip(out, meta):
            plain_seen += int(row[28])
            n_el += 1
            want_vals, want_grad = oracle_element(ga, gb, ea, eb, qA, tA, hA, tau, ybar, cls=2)
            e = element_errors(row[:18], want_vals, row[18:28], want_grad)
            assert within_bar(e), e
    assert plain_seen == n_el
