"""Shared helpers of the GPU-vs-oracle parity tests.

The bar.  The FP32 path is held to the fixed absolute tolerance TOL (1e-5 on
contact points and signed distances, 1e-4 on normals and weights; gradients 1e-3
relative to each pair's largest component).  A pair that misses it is held
instead to its own conditioning: the FP64 oracle is evaluated again at the
pair's FP32 inputs each moved by one ulp (every pose, dimension, tau, vertex and
plane entry independently, random sign; ULP_DRAWS draws), and the pair passes if
every field is within BOUND_FACTOR times the largest move of the oracle's own
output.  An FP32 evaluation rounds every input and every intermediate, so no
FP32 path can be held closer to the FP64 result than the inputs' rounding alone
moves it; BOUND_FACTOR allows for the ~10-100 roundings along the longest
dependency chain of a candidate (SDF LSE over up to 500 planes, the 2x2 QP, the
indicators, the SoftSort), each of at most one ulp (two for the MUFU
approximations), adding up like a random walk: sqrt(100) x 1.6 = 16.
At tau = 1e-3 this matters: the soft sign, penetration and nearest-neighbour
indicators scale rounding by 1/tau and the SoftSort at temperature tau scales
the score error by 1/tau again, so a one-ulp move of the inputs alone moves some
pairs' oracle output by ~1e-4 (measured), ten times TOL.
"""
import numpy as np
import torch

import oracle
import synth

# Tolerances of the FP32 GPU path against the FP64 oracle (unit-scale geometry):
# absolute 1e-5 on contact points and signed distances, 1e-4 on normals.  The
# activity weight w lies in [0, 1] and is held to 1e-4 absolute as well.
TOL = {"p": 1e-5, "d": 1e-5, "n": 1e-4, "w": 1e-4}
SLICES = {"p": slice(0, 3), "d": slice(3, 4), "n": slice(4, 7), "w": slice(7, 8)}
GRAD_REL = 1e-3
BOUND_FACTOR = 16.0
ULP_DRAWS = 4


def oracle_params(p):
    return oracle.Params(K=p.K, w_reg=p.w_reg, eps_clip=p.eps_clip, eps_min=p.eps_min,
                         eps_comp=p.eps_comp, no_ee=bool(p.flags & 1), one_sided=bool(p.flags & 2),
                         trace_iters=int(getattr(p, "trace_iters", 0)))


def _selects(params):
    return bool(getattr(params, "top_verts", 0) or getattr(params, "top_edges", 0))


def oracle_forward(w, params, idx=None):
    if _selects(params):
        return oracle_forward_preselect(w, params, idx)
    return oracle.batch_manifold(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau,
                                 oracle_params(params), idx=idx)


def oracle_forward_preselect(w, params, idx=None):
    from oracle.preselect import pair_manifold_preselect
    ids = range(w.n_pairs) if idx is None else idx
    t = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa: E731
    out = []
    with torch.no_grad():
        for i in ids:
            ga, gb = w.geoms[int(w.pair_geoms[i, 0])], w.geoms[int(w.pair_geoms[i, 1])]
            out.append(pair_manifold_preselect(ga, gb, t(w.poses[i]), t(w.dims[i]), float(w.tau[i]),
                                               oracle_params(params), params.top_verts, params.top_edges).numpy())
    return np.stack(out)


def oracle_grad(w, params, grad_out, idx=None, dtype=torch.float64):
    """dL/d (poses, dims) as (n, 20) by autograd through the oracle for upstream
    ``grad_out`` (n, K, 8) of the pairs ``idx`` (float64 is the reference; float32 only
    measures a plain FP32 evaluation of the same steps)."""
    ids = list(range(w.n_pairs)) if idx is None else [int(i) for i in idx]
    if not _selects(params) and dtype == torch.float64:
        gp, gd = oracle.batch_manifold_grad(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau, grad_out,
                                            oracle_params(params), idx=ids)
        return np.concatenate([gp, gd], 1)
    from oracle.preselect import pair_manifold_preselect
    t = lambda x: torch.as_tensor(np.asarray(x), dtype=dtype)  # noqa: E731
    out = np.zeros((len(ids), 20))
    for j, i in enumerate(ids):
        ga, gb = w.geoms[int(w.pair_geoms[i, 0])], w.geoms[int(w.pair_geoms[i, 1])]
        pose = t(w.poses[i]).requires_grad_(True)
        dm = t(w.dims[i]).requires_grad_(True)
        if _selects(params):
            m = pair_manifold_preselect(ga, gb, pose, dm, float(w.tau[i]), oracle_params(params),
                                        params.top_verts, params.top_edges)
        else:
            from oracle.manifold import pair_manifold
            m = pair_manifold(ga, gb, pose, dm, float(w.tau[i]), oracle_params(params))
        a, b = torch.autograd.grad(m, (pose, dm), t(grad_out[j]), allow_unused=True)
        out[j, :14] = a.double().numpy()
        out[j, 14:] = 0.0 if b is None else b.double().numpy()
    return out


# ----------------------------------------------------------------- one-ulp conditioning
def _ulp(a, rng):
    """Every entry of float32 array ``a`` moved by one ulp up or down (random sign)."""
    a = np.asarray(a, np.float32)
    up = np.nextafter(a, np.float32(np.inf))
    dn = np.nextafter(a, np.float32(-np.inf))
    return np.where(rng.integers(0, 2, a.shape) == 1, up, dn).astype(np.float32)


def _ulp_geometry(g, rng):
    v = np.array(g.verts, np.float32, copy=True)
    v[:, :3] = _ulp(v[:, :3], rng)           # the template column (cap sign / 0) stays exact
    p = _ulp(g.planes, rng) if len(g.planes) else np.array(g.planes, copy=True)
    return synth.Geometry(g.kind, np.array(g.dims, copy=True), v, np.array(g.edges, copy=True), p)


def nudged(w, idx, rng):
    """The pairs ``idx`` of ``w`` with every FP32 input moved by one ulp: a workload of
    len(idx) pairs, pair j naming geometries 2j (A) and 2j + 1 (B)."""
    geoms, pg = [], []
    for j, i in enumerate(idx):
        ga, gb = w.geoms[int(w.pair_geoms[i, 0])], w.geoms[int(w.pair_geoms[i, 1])]
        geoms += [_ulp_geometry(ga, rng), _ulp_geometry(gb, rng)]
        pg.append((2 * j, 2 * j + 1))
    idx = np.asarray(idx)
    return synth.Workload(w.name + "[ulp]", geoms, np.asarray(pg, np.int32), _ulp(w.poses[idx], rng),
                          _ulp(w.dims[idx], rng), _ulp(w.tau[idx], rng), w.K)


def forward_spread(w, params, idx, ref, draws=ULP_DRAWS, seed=0):
    """Per pair and field (n, 4: p, d, n, w): the largest move of the oracle's manifold
    over ``draws`` one-ulp draws of the pair's inputs (``ref``: its manifold at the inputs)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((len(idx), 4))
    for _ in range(draws):
        m = oracle_forward(nudged(w, idx, rng), params)
        for f, (k, s) in enumerate(SLICES.items()):
            out[:, f] = np.maximum(out[:, f], np.abs(m[..., s] - ref[..., s]).reshape(len(idx), -1).max(1))
    return out


def grad_spread(w, params, idx, grad_out, ref, draws=ULP_DRAWS, seed=0):
    """Per pair: the largest move of the oracle's gradient (all 20 components) over
    ``draws`` one-ulp draws of the pair's inputs, upstream ``grad_out`` kept."""
    rng = np.random.default_rng(seed)
    out = np.zeros(len(idx))
    for _ in range(draws):
        g = oracle_grad(nudged(w, idx, rng), params, grad_out)
        out = np.maximum(out, np.abs(g - ref).max(1))
    return out


# ----------------------------------------------------------------- checks
def errors(gpu, ref):
    return {k: float(np.abs(gpu[..., s] - ref[..., s]).max()) for k, s in SLICES.items()}


def pair_errors(gpu, ref):
    """(n, 4) largest absolute error per pair and field (p, d, n, w)."""
    n = gpu.shape[0]
    return np.stack([np.abs(gpu[..., s] - ref[..., s]).reshape(n, -1).max(1) for s in SLICES.values()], 1)


def assert_close(gpu, ref, tol=TOL, what=""):
    """Every pair within the fixed tolerance ``tol``."""
    assert np.isfinite(gpu).all(), f"{what}: non-finite GPU output"
    err = errors(gpu, ref)
    bad = {k: v for k, v in err.items() if v > tol[k]}
    if bad:
        worst = {}
        for k in bad:
            e = np.abs(gpu[..., SLICES[k]] - ref[..., SLICES[k]]).reshape(gpu.shape[0], -1).max(1)
            worst[k] = (int(np.argmax(e)), float(e.max()))
        raise AssertionError(f"{what}: errors {err} exceed {tol}; worst pair per field {worst}")
    return err


def assert_parity(gpu, ref, w, params, idx, what=""):
    """Every pair ``idx[j]`` (rows gpu[j], ref[j]) within TOL, or within BOUND_FACTOR times
    its one-ulp spread (module docstring).  Returns a summary: the worst errors, the share
    of pairs within TOL and, for the others, the largest error / spread ratio."""
    assert np.isfinite(gpu).all(), f"{what}: non-finite GPU output"
    idx = np.asarray(idx)
    e = pair_errors(gpu, ref)
    tol = np.array([TOL[k] for k in SLICES])
    over = (e > tol).any(1)
    info = {"pairs": len(idx), "within_tol": float(1.0 - over.mean()),
            "max_err": dict(zip(SLICES, e.max(0).tolist()))}
    if over.any():
        sub = np.nonzero(over)[0]
        spread = forward_spread(w, params, idx[sub], ref[sub])
        bound = np.maximum(tol, BOUND_FACTOR * spread)
        ratio = e[sub] / np.maximum(spread, 1e-300)
        info["bounded_by_spread"] = int(len(sub))
        info["max_err_over_spread"] = float(np.where(e[sub] > tol, ratio, 0.0).max())
        bad = (e[sub] > bound).any(1)
        if bad.any():
            j = sub[np.argmax(((e[sub] - bound) / bound).max(1))]
            k = int(np.nonzero(sub == j)[0][0])
            raise AssertionError(
                f"{what}: pair {int(idx[j])} (tau={float(w.tau[idx[j]]):g}) errors {dict(zip(SLICES, e[j]))} "
                f"exceed max(TOL, {BOUND_FACTOR} x one-ulp spread {dict(zip(SLICES, spread[k]))}); "
                f"{int(bad.sum())} of {len(idx)} pairs fail")
    return info


def assert_grad_parity(got, ref, w, params, idx, grad_out, what=""):
    """Every pair's gradient (n, 20) within GRAD_REL of its largest oracle component, or
    within BOUND_FACTOR times the oracle gradient's one-ulp spread."""
    assert np.isfinite(got).all(), f"{what}: non-finite gradient"
    idx = np.asarray(idx)
    scale = np.maximum(np.abs(ref).max(1), 1e-30)
    err = np.abs(got - ref).max(1)
    rel = err / scale
    over = rel > GRAD_REL
    info = {"pairs": len(idx), "within_rel": float(1.0 - over.mean()), "max_rel": float(rel.max())}
    if over.any():
        sub = np.nonzero(over)[0]
        spread = grad_spread(w, params, idx[sub], grad_out[sub], ref[sub])
        bound = np.maximum(GRAD_REL * scale[sub], BOUND_FACTOR * spread)
        info["bounded_by_spread"] = int(len(sub))
        info["max_err_over_spread"] = float((err[sub] / np.maximum(spread, 1e-300)).max())
        bad = err[sub] > bound
        if bad.any():
            j = int(np.argmax(err[sub] / bound))
            raise AssertionError(
                f"{what}: pair {int(idx[sub[j]])} (tau={float(w.tau[idx[sub[j]]]):g}) gradient error "
                f"{err[sub[j]]:.3g} (rel {rel[sub[j]]:.3g}) exceeds max({GRAD_REL} x {scale[sub[j]]:.3g}, "
                f"{BOUND_FACTOR} x one-ulp spread {spread[j]:.3g}); {int(bad.sum())} of {len(idx)} pairs fail")
    return info


def contact_share(w, idx, params=None, frac_tau=1.0):
    """Share of the pairs ``idx`` whose largest candidate score -w d exceeds frac_tau x tau
    in the oracle (pairs whose top SoftSort rows are active contacts)."""
    from oracle.manifold import pair_candidates
    p = oracle_params(params) if params is not None else oracle.Params()
    t = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa: E731
    hits = []
    with torch.no_grad():
        for i in idx:
            ga, gb = w.geoms[int(w.pair_geoms[i, 0])], w.geoms[int(w.pair_geoms[i, 1])]
            c = pair_candidates(ga, gb, t(w.poses[i]), t(w.dims[i]), float(w.tau[i]), p)
            hits.append(float((-c[:, 7] * c[:, 3]).max()) > frac_tau * float(w.tau[i]))
    return float(np.mean(hits))


def check_forward(gpu, w, params, idx=None, what=""):
    """The GPU rows ``gpu`` of pairs ``idx`` (default: all) against the oracle under the
    per-pair bar (assert_parity); prints and returns the summary."""
    idx = np.arange(w.n_pairs) if idx is None else np.asarray(idx)
    ref = oracle_forward(w, params, idx=idx)
    info = assert_parity(np.asarray(gpu, np.float64), ref, w, params, idx, what)
    print(what, info)
    return info


def check_grad(got, w, params, grad_out, idx=None, what=""):
    """GPU gradients ``got`` (n, 20) of pairs ``idx`` for upstream ``grad_out`` against the
    oracle's autograd under the per-pair bar (assert_grad_parity)."""
    idx = np.arange(w.n_pairs) if idx is None else np.asarray(idx)
    ref = oracle_grad(w, params, grad_out, idx=idx)
    info = assert_grad_parity(np.asarray(got, np.float64), ref, w, params, idx, np.asarray(grad_out), what)
    print(what, info)
    return info
