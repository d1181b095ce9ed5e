"""Write ``oracle_small.json``: a small stored case of the FP64 oracle.

Run from the repository root as ``python tests/golden/make_golden.py``.  Only
``synth`` (seeded inputs) and ``oracle`` are called; nothing here touches the
CUDA library.  The paper prints no worked numeric example, so these values are
the oracle's, not the paper's: they freeze the oracle's whole-manifold result
(Sec. IV-A candidates, Sec. IV-C V-S, Sec. IV-D E-E witnesses, Sec. III SoftSort
top-K) and its vector-Jacobian product on a dozen pairs, so that a change of
the oracle's arithmetic shows up as a failing CPU test and the CUDA path can be
compared with FP64 values without re-running the oracle.

With each pair it stores the pair's one-ulp conditioning (how far the oracle's
manifold and gradient move when every FP32 input of the pair moves by one ulp,
four draws; tests/_parity.py), so the GPU test applies the per-pair bar.

The case holds every input in full (the geometries used, the pair table,
poses, dimensions, smoothing and the upstream gradient), so it does not depend
on the generators staying unchanged:

* 4 box-box pairs of the resting-box workload (tau = 1e-2);
* for each primitive kind the pair of the hull-vs-primitive workload whose hull
  has the fewest vertices (tau = 1e-2), and the same four pairs at tau = 1e-1;
* one box-box pair moved 3 units apart along x (no contact: every activity
  weight near zero, the manifold still finite).
"""
import json
import os
import sys
from types import SimpleNamespace

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

sys.path.insert(0, os.path.dirname(HERE))
import _parity  # noqa: E402  (the one-ulp conditioning of the oracle, tests/_parity.py)

OUT = os.path.join(HERE, "oracle_small.json")
GRAD_SEED = 7


def build_case():
    """The inputs of the stored case as plain arrays (float32 where the library takes float32)."""
    bb = synth.make_config(1, 8)
    hp = synth.make_config(2, 256)
    npts = np.array([g.n_verts for g in hp.geoms])
    picks = []
    for k in synth.PRIMITIVE_KINDS:
        rows = np.nonzero(hp.pair_geoms[:, 1] == synth.PRIMITIVE_KINDS.index(k))[0]
        picks.append(int(rows[np.argmin(npts[hp.pair_geoms[rows, 0]])]))

    geoms, index = [], {}

    def gid(w, i):
        key = (w.name, int(i))
        if key not in index:
            index[key] = len(geoms)
            geoms.append(w.geoms[int(i)])
        return index[key]

    pg, poses, dims, tau = [], [], [], []

    def add(w, i, t=None, shift=0.0):
        pg.append((gid(w, w.pair_geoms[i, 0]), gid(w, w.pair_geoms[i, 1])))
        p = w.poses[i].copy()
        p[11] += np.float32(shift)
        poses.append(p)
        dims.append(w.dims[i].copy())
        tau.append(np.float32(w.tau[i] if t is None else t))

    for i in range(4):
        add(bb, i)
    for i in picks:
        add(hp, i)
    for i in picks:
        add(hp, i, t=1e-1)
    add(bb, 4, shift=3.0)
    rng = np.random.default_rng(GRAD_SEED)
    n = len(pg)
    grad_out = rng.standard_normal((n, 8, 8)).astype(np.float32)
    return (geoms, np.array(pg, np.int32), np.stack(poses).astype(np.float32),
            np.stack(dims).astype(np.float32), np.array(tau, np.float32), grad_out)


def geometry_to_dict(g):
    return {"kind": int(g.kind), "dims": np.asarray(g.dims, np.float64).tolist(),
            "verts": np.asarray(g.verts, np.float64).tolist(),
            "edges": np.asarray(g.edges, np.int64).tolist(),
            "planes": np.asarray(g.planes, np.float64).reshape(-1, 4).tolist()}


def geometry_from_dict(d):
    return synth.Geometry(kind=int(d["kind"]), dims=np.asarray(d["dims"], np.float32),
                          verts=np.asarray(d["verts"], np.float32).reshape(-1, 4),
                          edges=np.asarray(d["edges"], np.int32).reshape(-1, 2),
                          planes=np.asarray(d["planes"], np.float32).reshape(-1, 4))


def load(path=OUT):
    """The stored case as a dict of numpy arrays plus ``geoms`` (list of synth.Geometry)."""
    with open(path) as f:
        d = json.load(f)
    out = {k: np.asarray(v) for k, v in d.items() if k not in ("geoms", "params", "about")}
    out["geoms"] = [geometry_from_dict(g) for g in d["geoms"]]
    out["params"] = d["params"]
    out["about"] = d["about"]
    for k in ("poses", "dims", "tau", "grad_out"):
        out[k] = out[k].astype(np.float32)
    out["pair_geoms"] = out["pair_geoms"].astype(np.int32)
    return out


def main():
    geoms, pg, poses, dims, tau, grad_out = build_case()
    params = oracle.Params()
    manifold = oracle.batch_manifold(geoms, pg, poses, dims, tau, params)
    gp, gd = oracle.batch_manifold_grad(geoms, pg, poses, dims, tau, grad_out, params)
    # each pair's one-ulp conditioning (the per-pair bar of tests/_parity.py), so the GPU
    # test of this case applies the same bar without running the oracle
    w = synth.Workload("golden", geoms, pg, poses, dims, tau)
    idx = np.arange(len(pg))
    p = SimpleNamespace(K=params.K, w_reg=params.w_reg, eps_clip=params.eps_clip, eps_min=params.eps_min,
                        eps_comp=params.eps_comp, flags=0, top_verts=0, top_edges=0, trace_iters=0)
    fwd_spread = _parity.forward_spread(w, p, idx, manifold)
    grad_spread = _parity.grad_spread(w, p, idx, grad_out, np.concatenate([gp, gd], 1))
    doc = {
        "about": "FP64 oracle output on a small seeded case; written by tests/golden/make_golden.py "
                 "from oracle/ only (whole manifold: Sec. IV-A, IV-C, IV-D, Sec. III).",
        "params": {"K": params.K, "w_reg": params.w_reg, "eps_clip": params.eps_clip,
                   "eps_min": params.eps_min, "eps_comp": params.eps_comp, "flags": 0},
        "geoms": [geometry_to_dict(g) for g in geoms],
        "pair_geoms": pg.tolist(),
        "poses": poses.astype(np.float64).tolist(),
        "dims": dims.astype(np.float64).tolist(),
        "tau": tau.astype(np.float64).tolist(),
        "grad_out": grad_out.astype(np.float64).tolist(),
        "manifold": manifold.tolist(),
        "grad_poses": gp.tolist(),
        "grad_dims": gd.tolist(),
        "spread_fwd": fwd_spread.tolist(),
        "spread_grad": grad_spread.tolist(),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {OUT}: {len(pg)} pairs, {len(geoms)} geometries, {os.path.getsize(OUT)} bytes")


if __name__ == "__main__":
    main()
