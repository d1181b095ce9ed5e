"""Edge-edge witness points and E-E contact candidates (Sec. IV-D2, IV-D3; Supplement C).

Test infrastructure (see ``oracle/__init__``).

Witness points: points on edge j are e_j(a) = v_I + a (v_II - v_I), a in [0, 1].
With A = [t1, e2_I - e2_II] and b = e1_I - e2_I the distance is |A alpha + b|;
adding the L2 term lam [(a1 - 1/2)^2 + (a2 - 1/2)^2] (Sec. IV-D2) and halving
gives the box QP  min 1/2 alpha^T Q alpha + c^T alpha,  0 <= alpha <= 1,  with
Q = A^T A + lam I and c = A^T b - lam (1/2, 1/2).

The smoothed analytic active set (Sec. IV-D2, steps i-iv):
  i.   unconstrained minimiser alpha_u = -Q^-1 c (the text's "Q^-1 c" misses
       the sign of its own objective; read as -Q^-1 c);
  ii.  the four minimisers along the box edges a1 = 1, a1 = 0, a2 = 1, a2 = 0,
       each the 1-D stationary point soft-clipped to [0, 1] (the text's
       "-(Q12 - c2)/Q22" for the edge a1 = 1 is read as -(Q12 + c2)/Q22, the
       stationary point of the objective), their objective values, and the
       soft-argmin blend alpha_c of the four;
  iii. con = within_s(alpha_u1) * within_s(alpha_u2);
  iv.  alpha* = con alpha_u + (1 - con) alpha_c.
Every objective value is the objective itself evaluated at the candidate, so
the four costs are mutually consistent (this is what makes the solve
equivariant under swapping the two edges).

Non-smoothed variant (the paper's Ours-NS, Sec. V): the same steps with the
hard operators -- the side minimisers clipped to [0, 1], the argmin of the four
costs (first on ties), con the Iverson bracket of 0 <= alpha_u <= 1 in both
coordinates (inclusive) and alpha* = alpha_u where con, else the argmin side's
point.  For the strictly convex regularised QP this is the exact minimiser over
the box (interior minimiser if feasible, else the best of the four sides, each
minimised exactly by clipping its 1-D stationary point).

Pins: tests/test_oracle_edge_edge.py -- dense-grid brute force of the
regularised QP in the near-hard limit and of the non-smoothed solve, the skew-perpendicular closed form,
the parallel-edges closed form, swap equivariance, and continuity of the
rotating-edge sweep of Fig. 4 (with a jump when smoothing is switched off).
"""
import torch

from .smooth import argmin_s, clip_s, sigmoid, within_s


def _objective(Q11, Q12, Q22, c1, c2, a1, a2):
    return 0.5 * (Q11 * a1 * a1 + 2.0 * Q12 * a1 * a2 + Q22 * a2 * a2) + c1 * a1 + c2 * a2


def solve_box_qp(Q11, Q12, Q22, c1, c2, eps_clip=0.1, eps_min=0.1, eps_comp=0.1):
    """Smoothed analytic active-set solve of the 2x2 box QP.  Returns (a1, a2, con)."""
    det = Q11 * Q22 - Q12 * Q12
    a1_u = (Q12 * c2 - Q22 * c1) / det
    a2_u = (Q12 * c1 - Q11 * c2) / det
    one, zero = torch.ones_like(a1_u), torch.zeros_like(a1_u)
    # minimisers along the four sides of the unit box
    s1 = clip_s(-(Q12 + c2) / Q22, 0.0, 1.0, eps_clip)   # a1 = 1
    s2 = clip_s(-c2 / Q22, 0.0, 1.0, eps_clip)           # a1 = 0
    s3 = clip_s(-(Q12 + c1) / Q11, 0.0, 1.0, eps_clip)   # a2 = 1
    s4 = clip_s(-c1 / Q11, 0.0, 1.0, eps_clip)           # a2 = 0
    a1_c = torch.stack([one, zero, s3, s4], dim=-1)
    a2_c = torch.stack([s1, s2, one, zero], dim=-1)
    costs = _objective(Q11[..., None], Q12[..., None], Q22[..., None],
                       c1[..., None], c2[..., None], a1_c, a2_c)
    prob = argmin_s(costs, eps_min, dim=-1)
    a1_cb = (prob * a1_c).sum(-1)
    a2_cb = (prob * a2_c).sum(-1)
    con = within_s(a1_u, 0.0, 1.0, eps_comp) * within_s(a2_u, 0.0, 1.0, eps_comp)
    a1 = con * a1_u + (1.0 - con) * a1_cb
    a2 = con * a2_u + (1.0 - con) * a2_cb
    return a1, a2, con


def solve_box_qp_hard(Q11, Q12, Q22, c1, c2):
    """Non-smoothed analytic active-set solve (Ours-NS).  Returns (a1, a2, con)."""
    det = Q11 * Q22 - Q12 * Q12
    a1_u = (Q12 * c2 - Q22 * c1) / det
    a2_u = (Q12 * c1 - Q11 * c2) / det
    one, zero = torch.ones_like(a1_u), torch.zeros_like(a1_u)
    s1 = torch.clamp(-(Q12 + c2) / Q22, 0.0, 1.0)   # a1 = 1
    s2 = torch.clamp(-c2 / Q22, 0.0, 1.0)           # a1 = 0
    s3 = torch.clamp(-(Q12 + c1) / Q11, 0.0, 1.0)   # a2 = 1
    s4 = torch.clamp(-c1 / Q11, 0.0, 1.0)           # a2 = 0
    a1_c = torch.stack([one, zero, s3, s4], dim=-1)
    a2_c = torch.stack([s1, s2, one, zero], dim=-1)
    costs = _objective(Q11[..., None], Q12[..., None], Q22[..., None],
                       c1[..., None], c2[..., None], a1_c, a2_c)
    j = torch.argmin(costs, dim=-1, keepdim=True)
    a1_cb = torch.gather(a1_c, -1, j)[..., 0]
    a2_cb = torch.gather(a2_c, -1, j)[..., 0]
    inside = (a1_u >= 0.0) & (a1_u <= 1.0) & (a2_u >= 0.0) & (a2_u <= 1.0)
    return torch.where(inside, a1_u, a1_cb), torch.where(inside, a2_u, a2_cb), inside.to(a1_u.dtype)


def ee_witness(a0, a1, b0, b1, w_reg=0.01, eps_clip=0.1, eps_min=0.1, eps_comp=0.1, hard=False):
    """Witness points of edge pairs (a0, a1) x (b0, b1) (broadcasting, (..., 3)); with
    ``hard`` the non-smoothed solve (Ours-NS).

    Returns (e1*, e2*, alpha1, alpha2, con).
    """
    t1 = a1 - a0
    t2 = b0 - b1
    b = a0 - b0
    Q11 = (t1 * t1).sum(-1) + w_reg
    Q12 = (t1 * t2).sum(-1)
    Q22 = (t2 * t2).sum(-1) + w_reg
    c1 = (t1 * b).sum(-1) - 0.5 * w_reg
    c2 = (t2 * b).sum(-1) - 0.5 * w_reg
    if hard:
        al1, al2, con = solve_box_qp_hard(Q11, Q12, Q22, c1, c2)
    else:
        al1, al2, con = solve_box_qp(Q11, Q12, Q22, c1, c2, eps_clip, eps_min, eps_comp)
    e1 = a0 + al1[..., None] * (a1 - a0)
    e2 = b0 + al2[..., None] * (b1 - b0)
    return e1, e2, al1, al2, con


def _norm(v):
    r2 = (v * v).sum(-1)
    pos = r2 > 0
    r = torch.sqrt(torch.where(pos, r2, torch.ones_like(r2)))
    return torch.where(pos, r, torch.zeros_like(r))


def trace_to_surface(x, sdf, iters):
    """Sphere tracing of points x (..., 3) onto the zero set of ``sdf`` (Supplement,
    mesh-SDF discrepancies): the direction is fixed at the start point, u = grad phi(x_0)
    / |grad phi(x_0)|, and each of ``iters`` steps moves x <- x - phi(x) u."""
    phi, nu = sdf(x)
    u = nu / torch.linalg.vector_norm(nu, dim=-1, keepdim=True)
    for i in range(iters):
        if i:
            phi, _ = sdf(x)
        x = x - phi[..., None] * u
    return x


def ee_candidates(a0, a1, b0, b1, sdfA, sdfB, tau, w_reg=0.01, eps_clip=0.1, eps_min=0.1,
                  eps_comp=0.1, trace_iters=0):
    """All E-E contact candidates of one body pair (Sec. IV-D3).

    a0, a1: (E_A, 3) world endpoints of A's edges; b0, b1: (E_B, 3) of B's.
    sdfA / sdfB: callables world points -> (phi, world normal) of each body.
    Returns dict of (E_A, E_B[, 3]) tensors for witness 1 (on A) and 2 (on B):
    p1, d1, n1, w1, p2, d2, n2, w2, plus the intermediate indicators.

    Sign (Sec. IV-D3): witness b uses its own offset from the other witness,
    dbar_b = e_b* - e_o*, and the other body's normal at e_o*:
    gamma_b = tanh(nu_o(e_o*) . nbar_b / tau).  (The text's "vice versa" with one
    shared nbar would make a penetrating witness on B positive; this reading
    makes both penetrating witnesses negative and the whole manifold symmetric
    under swapping A and B.)  eps in nbar = Delta / sqrt(|Delta|^2 + eps) is tau^2.
    Soft-sign and nearest-neighbour softmax use temperature tau.

    trace_iters > 0 projects each witness onto its own body's SDF surface first
    (trace_to_surface, e1* on A and e2* on B) and the signed distances, normals,
    penetration and clash indicators and the output points use the projected
    witnesses.  The nearest-neighbour indicators stay on the QP witnesses' own
    distances (reading: the supplement moves the points used for signed
    distances and normals; the nn softmax ranks edge pairs).
    """
    e1, e2, al1, al2, con = ee_witness(a0[:, None, :], a1[:, None, :], b0[None, :, :],
                                       b1[None, :, :], w_reg, eps_clip, eps_min, eps_comp)
    dbar_qp = _norm(e1 - e2)
    if trace_iters:
        e1 = trace_to_surface(e1, sdfA, trace_iters)
        e2 = trace_to_surface(e2, sdfB, trace_iters)
    delta = e1 - e2
    dbar = _norm(delta)
    nbar1 = delta / torch.sqrt((delta * delta).sum(-1, keepdim=True) + tau * tau)
    nbar2 = -nbar1
    phiB_e1, _ = sdfB(e1)          # penetration of witness 1 into B
    phiA_e2, _ = sdfA(e2)          # penetration of witness 2 into A
    _, nuA_e1 = sdfA(e1)           # A's normal at witness 1
    _, nuB_e2 = sdfB(e2)           # B's normal at witness 2
    g1 = torch.tanh((nuB_e2 * nbar1).sum(-1) / tau)
    g2 = torch.tanh((nuA_e1 * nbar2).sum(-1) / tau)
    pen1 = sigmoid(-phiB_e1 / tau)
    pen2 = sigmoid(-phiA_e2 / tau)
    cl = sigmoid(-(nuA_e1 * nuB_e2).sum(-1) / tau)
    nn1 = torch.softmax(-dbar_qp / tau, dim=1)    # row-wise over B's edges
    nn2 = torch.softmax(-dbar_qp / tau, dim=0)    # column-wise over A's edges
    w1 = con * pen1 * nn1 * cl
    w2 = con * pen2 * nn2 * cl
    return dict(p1=e1, d1=g1 * dbar, n1=g1[..., None] * nbar1, w1=w1,
                p2=e2, d2=g2 * dbar, n2=g2[..., None] * nbar2, w2=w2,
                dbar=dbar, con=con, pen1=pen1, pen2=pen2, cl=cl, nn1=nn1, nn2=nn2,
                alpha1=al1, alpha2=al2, gamma1=g1, gamma2=g2)
