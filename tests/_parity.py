"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

import oracle

# Tolerances of the FP32 GPU path against the FP64 oracle (unit-scale geometry):
# absolute 1e-5 on contact points and signed distances, 1e-4 on normals.  The
# activity weight w lies in [0, 1] and is held to 1e-4 absolute as well.
TOL = {"p": 1e-5, "d": 1e-5, "n": 1e-4, "w": 1e-4}
SLICES = {"p": slice(0, 3), "d": slice(3, 4), "n": slice(4, 7), "w": slice(7, 8)}


def tol_for_tau(tau):
    """Tolerance of the FP32 path at smoothing ``tau``.

    tau >= 1e-2: the fixed absolute tolerance TOL.  Below 1e-2 the manifold's
    sensitivity to FP32-level perturbations grows like 1/tau^2 (the soft sign,
    penetration and nearest-neighbour indicators scale rounding by 1/tau, and
    the SoftSort at temperature tau scales the resulting score error by 1/tau
    again): a one-ulp relative perturbation of the FP32 inputs already moves the
    FP64 oracle's output by ~1e-4 at tau = 1e-3.  There the tolerance is the
    fixed one scaled by 2 (1e-2 / tau)^2, i.e. 2e-3 on p and d at tau = 1e-3.
    """
    if tau >= 1e-2:
        return dict(TOL)
    f = 2.0 * (1e-2 / tau) ** 2
    return {k: v * f for k, v in TOL.items()}


def oracle_params(p):
    return oracle.Params(K=p.K, w_reg=p.w_reg, eps_clip=p.eps_clip, eps_min=p.eps_min,
                         eps_comp=p.eps_comp, no_ee=bool(p.flags & 1), one_sided=bool(p.flags & 2),
                         trace_iters=int(getattr(p, "trace_iters", 0)))


def oracle_forward(w, params, idx=None):
    if getattr(params, "top_verts", 0) or getattr(params, "top_edges", 0):
        return oracle_forward_preselect(w, params, idx)
    return oracle.batch_manifold(w.geoms, w.pair_geoms, w.poses, w.dims, w.tau,
                                 oracle_params(params), idx=idx)


def oracle_forward_preselect(w, params, idx=None):
    import torch
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


def errors(gpu, ref):
    return {k: float(np.abs(gpu[..., s] - ref[..., s]).max()) for k, s in SLICES.items()}


def assert_close(gpu, ref, tol=TOL, what=""):
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
