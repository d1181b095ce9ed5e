"""Soft top-K pre-selection of vertices and edges (Sec. IV-A; Supplement B).

Test infrastructure (see ``oracle/__init__``).

Before contacts are generated, every vertex gets a penetration metric from the
other body's SDF, m_v = phi_other(v), and every edge the weighted sum of its
corner metrics, m_e = (m_i + m_j) / 2 (equal weights: reading).  A soft top-K
over the depths -m (SoftSort, Sec. III, temperature tau: reading) gives K soft
indices Gamma_K; the selected vertices are Gamma_K V and the selected edges
(Gamma_K E_1, Gamma_K E_2), the soft averages of the edges' first and second
endpoints.  V-S contacts then use the selected vertices and E-E contacts the
K_A x K_B selected edge pairs.  The safeguard of Supplement B scales each E-E
witness's activity by the soft indicator that it lies inside its own body,
sigmoid(-phi_b(e_b*) / tau).  ``top_verts`` / ``top_edges`` of 0 keep all.

Pins: tests/test_oracle_preselect.py -- selection in the hard limit picks the
deepest vertices / edges, soft-index rows sum to one, edge metrics are the
corner averages, and with everything selected in the hard limit (safeguard
off) the manifold equals the unselected one.
"""
import torch

from .edge_edge import ee_candidates
from .manifold import _Body, soft_topk_reduce


def soft_select(score, values, K, tau):
    """SoftSort soft indices of the K largest scores applied to ``values`` (N, C) -> (K, C)."""
    top = torch.topk(score, K, largest=True, sorted=True).values
    gamma = torch.softmax(-torch.abs(top[:, None] - score[None, :]) / tau, dim=1)
    return gamma @ values, gamma


def pair_candidates_preselect(geomA, geomB, pose, dims, tau, params, top_verts=0, top_edges=0,
                              safeguard=True, tau_sel=None):
    """Candidate rows (N, 8) of one pair with soft pre-selection."""
    tsel = tau if tau_sel is None else tau_sel
    A = _Body(geomA, pose[:7], dims[:3], tau)
    B = _Body(geomB, pose[7:], dims[3:], tau)
    mA, _ = B.sdf(A.verts)
    mB, _ = A.sdf(B.verts)
    rows = []
    for own, other, m in ((A, B, mA), (B, A, mB)):
        verts = own.verts
        if top_verts:
            verts, _ = soft_select(-m, own.verts, min(top_verts, len(m)), tsel)
        phi, nu = other.sdf(verts)
        w = torch.sigmoid(-phi / tau)
        rows.append(torch.cat([verts, phi[:, None], nu, w[:, None]], dim=1))
    ends = []
    for own, m in ((A, mA), (B, mB)):
        e0, e1 = own.verts[own.edges[:, 0]], own.verts[own.edges[:, 1]]
        if top_edges:
            me = 0.5 * (m[own.edges[:, 0]] + m[own.edges[:, 1]])
            sel, _ = soft_select(-me, torch.cat([e0, e1], dim=1), min(top_edges, len(me)), tsel)
            e0, e1 = sel[:, :3], sel[:, 3:]
        ends.append((e0, e1))
    (a0, a1), (b0, b1) = ends
    c = ee_candidates(a0, a1, b0, b1, A.sdf, B.sdf, tau, params.w_reg, params.eps_clip, params.eps_min,
                      params.eps_comp, params.trace_iters)
    w1, w2 = c["w1"], c["w2"]
    if safeguard:
        phiA_e1, _ = A.sdf(c["p1"])
        phiB_e2, _ = B.sdf(c["p2"])
        w1 = w1 * torch.sigmoid(-phiA_e1 / tau)
        w2 = w2 * torch.sigmoid(-phiB_e2 / tau)
    for j, w in ((1, w1), (2, w2)):
        p, d, n = c[f"p{j}"], c[f"d{j}"], c[f"n{j}"]
        rows.append(torch.cat([p.reshape(-1, 3), d.reshape(-1, 1), n.reshape(-1, 3), w.reshape(-1, 1)], dim=1))
    return torch.cat(rows, dim=0)


def pair_manifold_preselect(geomA, geomB, pose, dims, tau, params, top_verts=0, top_edges=0,
                            safeguard=True, tau_sel=None):
    """(K, 8) manifold of one pair with soft pre-selection of vertices and edges."""
    cand = pair_candidates_preselect(geomA, geomB, pose, dims, tau, params, top_verts, top_edges,
                                     safeguard, tau_sel)
    return soft_topk_reduce(cand, tau, params.K)
