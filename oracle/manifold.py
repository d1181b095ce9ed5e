"""Whole contact manifold of a body pair and its K-point reduction (Sec. IV-A, IV-C, IV-D; Sec. III).

Test infrastructure (see ``oracle/__init__``).

Candidates of a pair (A, B), all in world coordinates (Sec. IV-A):
* V-S (Sec. IV-C): every vertex v of A gives (p = v, d = phi_B(v),
  n = nu_B(v), w = sigmoid(-d / tau)); every vertex of B likewise against A.
  The paper does not define a V-S activity; sigmoid(-d / tau) mirrors the
  penetration indicator of the E-E routine (reading).
* E-E (Sec. IV-D): every edge pair (k, l) gives two witnesses (oracle/edge_edge).

Reduction (reading): scores s_i = -w_i d_i; s^_1 >= ... >= s^_K are the K
largest scores; the SoftSort rows Gamma_{k,i} = softmax_i(-|s^_k - s_i| / tau)
(Sec. III, SoftSort top-K) select the outputs
out_k = sum_i Gamma_{k,i} (p_i, d_i, n_i, w_i), a (K, 8) array per pair laid out
(p_x, p_y, p_z, d, n_x, n_y, n_z, w).  Parity of this step is unpinned by the
paper's own numbers; tests pin its limits (hard top-K as tau -> 0, rows that
sum to one, uniform rows for equal scores), its exact weights on two score
levels tau ln 3 apart, its independence of candidate order, and the
swap/rigid-motion invariances of the whole manifold.
"""
import dataclasses

import numpy as np
import torch

from .edge_edge import ee_candidates
from .sdf import local_vertices, quat_to_rot, sdf_world

F64 = torch.float64


@dataclasses.dataclass
class Params:
    K: int = 8
    w_reg: float = 0.01
    eps_clip: float = 0.1
    eps_min: float = 0.1
    eps_comp: float = 0.1
    no_ee: bool = False        # V-S contacts only
    one_sided: bool = False    # only A's vertices against B's SDF (implies no_ee)
    trace_iters: int = 0       # sphere-tracing steps for E-E witnesses (0 = off)


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=F64)


class _Body:
    """A posed body.  Its geometry takes the dtype of ``pose`` (float64 everywhere in the
    parity path; float32 only where a test measures how a plain FP32 evaluation of these
    same steps deviates)."""

    def __init__(self, geom, pose, dims, tau):
        self.kind = int(geom.kind)
        self.R = quat_to_rot(pose[:4])
        self.t = pose[4:7]
        self.dims = dims
        self.planes = torch.as_tensor(np.asarray(geom.planes), dtype=pose.dtype)
        self.edges = torch.as_tensor(np.asarray(geom.edges), dtype=torch.long)
        vloc = local_vertices(self.kind, torch.as_tensor(np.asarray(geom.verts), dtype=pose.dtype), dims)
        self.verts = vloc @ self.R.T + self.t
        self.tau = tau

    def sdf(self, x):
        return sdf_world(self.kind, x, self.R, self.t, self.dims, self.planes, self.tau)


def pair_candidates(geomA, geomB, pose, dims, tau, params=Params()):
    """All candidates of one pair as (N, 8) rows (p, d, n, w).

    pose: (14,) float64 (qA, tA, qB, tB); dims: (6,) float64; tau: float.
    """
    A = _Body(geomA, pose[:7], dims[:3], tau)
    B = _Body(geomB, pose[7:], dims[3:], tau)
    rows = []
    sides = [(A, B)] if params.one_sided else [(A, B), (B, A)]
    for own, other in sides:
        phi, nu = other.sdf(own.verts)
        w = torch.sigmoid(-phi / tau)
        rows.append(torch.cat([own.verts, phi[:, None], nu, w[:, None]], dim=1))
    if not (params.no_ee or params.one_sided):
        a0, a1 = A.verts[A.edges[:, 0]], A.verts[A.edges[:, 1]]
        b0, b1 = B.verts[B.edges[:, 0]], B.verts[B.edges[:, 1]]
        c = ee_candidates(a0, a1, b0, b1, A.sdf, B.sdf, tau, params.w_reg, params.eps_clip,
                          params.eps_min, params.eps_comp, params.trace_iters)
        for j in (1, 2):
            p, d, n, w = c[f"p{j}"], c[f"d{j}"], c[f"n{j}"], c[f"w{j}"]
            rows.append(torch.cat([p.reshape(-1, 3), d.reshape(-1, 1), n.reshape(-1, 3),
                                   w.reshape(-1, 1)], dim=1))
    return torch.cat(rows, dim=0)


def soft_topk_reduce(cand, tau, K):
    """SoftSort top-K reduction of candidate rows (N, 8) to (K, 8) (Sec. III)."""
    s = -cand[:, 7] * cand[:, 3]
    top = torch.topk(s, K, largest=True, sorted=True).values
    logits = -torch.abs(top[:, None] - s[None, :]) / tau
    gamma = torch.softmax(logits, dim=1)
    return gamma @ cand


def pair_manifold(geomA, geomB, pose, dims, tau, params=Params()):
    """(K, 8) manifold of one pair in float64."""
    cand = pair_candidates(geomA, geomB, pose, dims, tau, params)
    return soft_topk_reduce(cand, tau, params.K)


def batch_manifold(geoms, pair_geoms, poses, dims, tau, params=Params(), idx=None):
    """(n, K, 8) float64 numpy manifold for the pairs ``idx`` (default: all)."""
    n = len(pair_geoms) if idx is None else len(idx)
    ids = range(len(pair_geoms)) if idx is None else idx
    out = np.zeros((n, params.K, 8))
    with torch.no_grad():
        for j, i in enumerate(ids):
            ga, gb = geoms[int(pair_geoms[i][0])], geoms[int(pair_geoms[i][1])]
            out[j] = pair_manifold(ga, gb, _t(poses[i]), _t(dims[i]), float(tau[i]),
                                   params).numpy()
    return out


def batch_manifold_grad(geoms, pair_geoms, poses, dims, tau, grad_out, params=Params(),
                        idx=None):
    """Vector-Jacobian product of the manifold: returns (d/d poses (n, 14), d/d dims (n, 6)).

    ``grad_out``: (n, K, 8) upstream gradient for the pairs ``idx``.
    """
    ids = list(range(len(pair_geoms))) if idx is None else list(idx)
    gp = np.zeros((len(ids), 14))
    gd = np.zeros((len(ids), 6))
    for j, i in enumerate(ids):
        ga, gb = geoms[int(pair_geoms[i][0])], geoms[int(pair_geoms[i][1])]
        pose = _t(poses[i]).requires_grad_(True)
        dm = _t(dims[i]).requires_grad_(True)
        out = pair_manifold(ga, gb, pose, dm, float(tau[i]), params)
        g_pose, g_dims = torch.autograd.grad(out, (pose, dm), _t(grad_out[j]),
                                             allow_unused=True)
        gp[j] = g_pose.numpy()
        gd[j] = 0.0 if g_dims is None else g_dims.numpy()
    return gp, gd
