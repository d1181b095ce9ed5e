"""Vertex-face witness point of the smoothed active set (Sec. IV-D1; Supplement C, V-F routine).

Test infrastructure (see ``oracle/__init__``).

The closest point of a triangle T = (T0, T1, T2) to a vertex v, smoothed the
way Sec. IV-D1 describes for a general convex polygon:
  i.   unconstrained minimiser: the projection of v on the triangle's plane;
  ii.  constrained minimisers: the projection of v on each of the three edges,
       the edge parameter soft-clipped to [0, 1]; the soft argmin of their
       distances to v blends them;
  iii. the soft indicator that the plane projection lies inside the triangle:
       the product of within_s over its three barycentric coordinates;
  iv.  the blend of (i) and (ii) by that indicator.
The printed routine clips the projection *length* onto the unit edge
direction to [0, 1], which equals the edge parameter only for unit-length
edges; here the edge parameter t = (v - Ta).(Tb - Ta) / |Tb - Ta|^2 is
clipped (reading).

Non-smoothed variant (the paper's Ours-NS, Sec. V): the edge parameters clipped
to [0, 1], the argmin of the three distances (first on ties), the Iverson
bracket of all three barycentric coordinates in [0, 1] (inclusive), and the
plane projection where inside, else the argmin edge's point: the exact closest
point of the triangle.

Pins: tests/test_oracle_vertex_face.py -- interior projections equal the foot
of the perpendicular, outside queries in the hard limit equal the brute-force
closest point of a dense triangle sampling, barycentric identities, and
invariance under relabelling the triangle's corners.
"""
import torch

from .smooth import argmin_s, clip_s, within_s


def _dot(a, b):
    return (a * b).sum(-1)


def vf_witness(v, t0, t1, t2, eps_clip=0.1, eps_min=0.1, eps_comp=0.1, hard=False):
    """Smoothed closest point of triangles (t0, t1, t2) to points v, all (..., 3); with
    ``hard`` the non-smoothed routine (Ours-NS).

    Returns (witness (..., 3), inside indicator (...,)).
    """
    corners = (t0, t1, t2)
    cand, cost = [], []
    for a, b in ((0, 1), (1, 2), (0, 2)):
        ta, tb = corners[a], corners[b]
        e = tb - ta
        t = _dot(v - ta, e) / _dot(e, e)
        s = torch.clamp(t, 0.0, 1.0) if hard else clip_s(t, 0.0, 1.0, eps_clip)
        q = ta + s[..., None] * e
        cand.append(q)
        cost.append(torch.linalg.vector_norm(v - q, dim=-1))
    cands = torch.stack(cand, -2)
    if hard:
        j = torch.argmin(torch.stack(cost, -1), dim=-1)
        p_c = torch.gather(cands, -2, j[..., None, None].expand(*j.shape, 1, 3))[..., 0, :]
    else:
        prob = argmin_s(torch.stack(cost, -1), eps_min, dim=-1)
        p_c = (prob[..., None] * cands).sum(-2)
    d10, d20 = t1 - t0, t2 - t0
    nb = torch.cross(d10, d20, dim=-1)
    area2 = torch.linalg.vector_norm(nb, dim=-1)
    n = nb / area2[..., None]
    rel = v - t0
    p = rel - _dot(rel, n)[..., None] * n                  # plane projection, relative to t0
    b2 = _dot(torch.cross(d10, p, dim=-1), n) / area2       # weight of t2
    b1 = _dot(torch.cross(p, d20, dim=-1), n) / area2       # weight of t1
    b0 = 1.0 - b1 - b2
    if hard:
        inside = ((b0 >= 0.0) & (b0 <= 1.0) & (b1 >= 0.0) & (b1 <= 1.0) & (b2 >= 0.0) & (b2 <= 1.0)).to(v.dtype)
    else:
        inside = within_s(b0, 0.0, 1.0, eps_comp) * within_s(b1, 0.0, 1.0, eps_comp) * \
            within_s(b2, 0.0, 1.0, eps_comp)
    p_u = t0 + p
    w = inside[..., None] * p_u + (1.0 - inside[..., None]) * p_c
    return w, inside
