// cm_adjoint.cuh -- hand-written reverse-mode adjoints of the per-candidate
// arithmetic in cm_math.cuh / cm_pair.cuh.
//
// Every function recomputes the forward quantities it needs (nothing of the
// forward is stored per candidate) and accumulates parameter adjoints into an
// Adj record: the relative pose (R_rel, t_rel) of A in B's frame and the dims
// of both bodies.  The per-pair epilogue chains these to the quaternions and
// translations of both bodies.
#pragma once

#include "cm_math.cuh"

namespace cm {

struct Adj {
  float R[9];  // d L / d R_rel
  V3 t;        // d L / d t_rel
  V3 dA, dB;   // d L / d dims of A and B
};

CM_HD void adj_zero(Adj& a) {
  for (int i = 0; i < 9; ++i) a.R[i] = 0.f;
  a.t = a.dA = a.dB = v3(0.f, 0.f, 0.f);
}
// R += u v^T
CM_HD void add_outer(float* R, V3 u, V3 v) {
  R[0] = fmaf(u.x, v.x, R[0]); R[1] = fmaf(u.x, v.y, R[1]); R[2] = fmaf(u.x, v.z, R[2]);
  R[3] = fmaf(u.y, v.x, R[3]); R[4] = fmaf(u.y, v.y, R[4]); R[5] = fmaf(u.y, v.z, R[5]);
  R[6] = fmaf(u.z, v.x, R[6]); R[7] = fmaf(u.z, v.y, R[7]); R[8] = fmaf(u.z, v.z, R[8]);
}

// ---------------------------------------------------------------- smooth operators
CM_HD float sigmoid_grad_from(float s) { return s * (1.f - s); }            // d sigmoid / dx
// clip_s(x, 0, 1) and its derivative from shared exponentials: with e0 = exp(-|x| / eps)
// and e1 = exp(-|x - 1| / eps) the value is max(x, 0) - max(x - 1, 0) + eps ln((1 + e0) / (1 + e1))
// and the derivative sigma(x / eps) - sigma((x - 1) / eps), sigma(u / eps) = (u >= 0 ? 1 : e) / (1 + e).
CM_HD float clip01_s_vg(float x, float inv_eps, float eps, float& grad) {
  const float k = inv_eps * kLog2e;
  const float e0 = ex2(-fabsf(x) * k), e1 = ex2(-fabsf(x - 1.f) * k);
  const float r0 = rcp(1.f + e0), r1 = rcp(1.f + e1);
  grad = (x >= 0.f ? r0 : e0 * r0) - (x >= 1.f ? r1 : e1 * r1);
  return fmaxf(x, 0.f) - fmaxf(x - 1.f, 0.f) + (eps * kLn2) * lg2((1.f + e0) * r1);
}
// within01(x) = sigma(x / eps) sigma((1 - x) / eps) and its derivative
// within01 (sigma((1 - x) / eps) - sigma(x / eps)) / eps from the same two sigmoids.
CM_HD float within01_vg(float x, float inv_eps, float& grad) {
  const float a = sigmoid(x * inv_eps), b = sigmoid((1.f - x) * inv_eps);
  const float w = a * b;
  grad = w * (b - a) * inv_eps;
  return w;
}

// ---------------------------------------------------------------- normal
// nu = g / sqrt(tau + |g|^2)  ->  gbar
CM_HD V3 normal_bwd(V3 g, float tau, V3 nubar) {
  float r = rsq(tau + dot(g, g));
  float gn = dot(g, nubar);
  return nubar * r - g * (gn * r * r * r);
}

// ---------------------------------------------------------------- SDF primitives
// Each takes the forward (phi, g) at y and the adjoints (phibar, gbar) and
// accumulates ybar and (where the primitive depends on them) dbar.

// Box: planes +-e_i . y - h_i; pi_f = exp((s_f - phi)/tau); sbar_f = pi_f (phibar + gbar.(n_f - g)/tau).
CM_HD void sdf_box_bwd(V3 y, V3 h, const Sdf& f, float inv_tau, float phibar, V3 gbar, V3& ybar, V3& hbar) {
  const float k = inv_tau * kLog2e;
  const float yy[3] = {y.x, y.y, y.z}, hh[3] = {h.x, h.y, h.z}, gg[3] = {f.g.x, f.g.y, f.g.z},
              gb[3] = {gbar.x, gbar.y, gbar.z};
  const float gdotg = dot(gbar, f.g);
  float yb[3], hb[3];
  for (int i = 0; i < 3; ++i) {
    // plane +e_i: value y_i - h_i, normal e_i;  plane -e_i: value -y_i - h_i, normal -e_i
    float pp = ex2((yy[i] - hh[i] - f.phi) * k), pn = ex2((-yy[i] - hh[i] - f.phi) * k);
    float sp = pp * (phibar + (gb[i] - gdotg) * inv_tau);
    float sn = pn * (phibar + (-gb[i] - gdotg) * inv_tau);
    yb[i] = sp - sn;
    hb[i] = -(sp + sn);
    (void)gg;
  }
  ybar += v3(yb[0], yb[1], yb[2]);
  hbar += v3(hb[0], hb[1], hb[2]);
}

// Planes arrive pre-scaled by k = log2(e) / tau (see sdf_planes): the scaled
// plane value is the base-2 exponent and the unit normal is (k n) / k.
CM_HD void sdf_planes_bwd(V3 y, const float4* P, int nP, const Sdf& f, float inv_tau, float phibar, V3 gbar,
                          V3& ybar) {
  const float k = inv_tau * kLog2e, ik = rcp(k);
  const float base = phibar - dot(gbar, f.g) * inv_tau;
  const float mk = f.phi * k;
  const float gk = inv_tau * ik;  // gbar . n_f / tau with n_f = (k n_f) / k
  V3 acc = v3(0.f, 0.f, 0.f);
  for (int i = 0; i < nP; ++i) {
    float4 p = P[i];
    float s = fmaf(p.x, y.x, fmaf(p.y, y.y, fmaf(p.z, y.z, -p.w)));
    float pi = ex2(s - mk);
    float sb = pi * (base + (gbar.x * p.x + gbar.y * p.y + gbar.z * p.z) * gk);
    acc.x = fmaf(sb, p.x, acc.x);
    acc.y = fmaf(sb, p.y, acc.y);
    acc.z = fmaf(sb, p.z, acc.z);
  }
  ybar += acc * ik;
}

// Ellipsoid: phi = r - r f^-1/2, r = |y|, f = sum y_i^2/d_i^2; g = 2 y / d^2.
CM_HD void sdf_ellipsoid_bwd(V3 y, V3 d, float phibar, V3 gbar, V3& ybar, V3& dbar) {
  V3 id = v3(rcp(d.x), rcp(d.y), rcp(d.z));
  V3 yt = v3(y.x * id.x, y.y * id.y, y.z * id.z);
  float f = dot(yt, yt);
  float r2 = dot(y, y);
  float ir = r2 > 0.f ? rsq(r2) : 0.f;
  float r = r2 * ir;
  float fm12 = rsq(f);
  float fm32 = fm12 * fm12 * fm12;
  // d phi / d y = (1 - f^-1/2) y / r + r f^-3/2 y / d^2
  float a = (1.f - fm12) * ir, b = r * fm32;
  V3 dpdy = v3(y.x * (a + b * id.x * id.x), y.y * (a + b * id.y * id.y), y.z * (a + b * id.z * id.z));
  // d phi / d d_i = -r f^-3/2 y_i^2 / d_i^3
  V3 dpdd = v3(-b * yt.x * yt.x * id.x, -b * yt.y * yt.y * id.y, -b * yt.z * yt.z * id.z);
  // g_i = 2 y_i / d_i^2: dg_i/dy_i = 2 / d_i^2, dg_i/dd_i = -4 y_i / d_i^3
  ybar += v3(phibar * dpdy.x + 2.f * gbar.x * id.x * id.x, phibar * dpdy.y + 2.f * gbar.y * id.y * id.y,
             phibar * dpdy.z + 2.f * gbar.z * id.z * id.z);
  dbar += v3(phibar * dpdd.x - 4.f * gbar.x * yt.x * id.x * id.x, phibar * dpdd.y - 4.f * gbar.y * yt.y * id.y * id.y,
             phibar * dpdd.z - 4.f * gbar.z * yt.z * id.z * id.z);
}

// Capsule (rad, h): c = clip_s(z, -h, h); w = (x, y, z - c); rho = |w|; phi = rho - rad;
// g = (u_x, u_y, u_z (1 - c')) with u = w / rho, c' = sig+ - sig-.
CM_HD void sdf_capsule_bwd(V3 y, float rad, float h, float tau, float inv_tau, float phibar, V3 gbar, V3& ybar,
                           V3& dbar) {
  // the soft clip's softplus terms and sigmoids from shared exponentials (as in sdf_capsule)
  float up = (y.z + h) * inv_tau, dn = (y.z - h) * inv_tau;
  const float Eu = exp_(-fabsf(up)), Ed = exp_(-fabsf(dn));
  const float iu = rcp(1.f + Eu), id = rcp(1.f + Ed);
  float c = -h + tau * ((fmaxf(up, 0.f) - fmaxf(dn, 0.f)) + kLn2 * lg2((1.f + Eu) * id));
  float sp = up >= 0.f ? iu : Eu * iu, sn = dn >= 0.f ? id : Ed * id;
  float cp = sp - sn;
  V3 w = v3(y.x, y.y, y.z - c);
  float r2 = dot(w, w);
  float ir = r2 > 0.f ? rsq(r2) : 0.f;
  V3 u = w * ir;
  // g = (u_x, u_y, u_z (1 - c'))
  V3 ub = v3(gbar.x, gbar.y, gbar.z * (1.f - cp));
  float cpb = -gbar.z * u.z;
  // w adjoint: phi = |w| and u = w / |w|
  float uu = dot(u, ub);
  V3 wb = u * phibar + (ub - u * uu) * ir;
  // w = (x, y, z - c)
  float cb = -wb.z;
  float dcdz = cp, dcdh = -1.f + sp + sn;
  float gp = sigmoid_grad_from(sp), gn = sigmoid_grad_from(sn);
  float dcpdz = (gp - gn) * inv_tau, dcpdh = (gp + gn) * inv_tau;
  ybar += v3(wb.x, wb.y, wb.z + cb * dcdz + cpb * dcpdz);
  dbar += v3(-phibar, cb * dcdh + cpb * dcpdh, 0.f);
}

// Cylinder (rad, h): s = (rho - rad, z - h, -z - h), phi = LSE_tau(s), pi = softmax(s / tau),
// g = (pi0 x / rho, pi0 y / rho, pi1 - pi2).
CM_HD void sdf_cylinder_bwd(V3 y, float rad, float h, const Sdf& f, float inv_tau, float phibar, V3 gbar,
                            V3& ybar, V3& dbar) {
  float rho2 = y.x * y.x + y.y * y.y;
  float irho = rho2 > 0.f ? rsq(rho2) : 0.f;
  float rho = rho2 * irho;
  float k = inv_tau * kLog2e;
  float s0 = rho - rad, s1 = y.z - h, s2 = -y.z - h;
  float p0 = ex2((s0 - f.phi) * k), p1 = ex2((s1 - f.phi) * k), p2 = ex2((s2 - f.phi) * k);
  float ex = y.x * irho, ey = y.y * irho;
  float pb0 = gbar.x * ex + gbar.y * ey, pb1 = gbar.z, pb2 = -gbar.z;
  float m = pb0 * p0 + pb1 * p1 + pb2 * p2;
  float sb0 = phibar * p0 + p0 * (pb0 - m) * inv_tau;
  float sb1 = phibar * p1 + p1 * (pb1 - m) * inv_tau;
  float sb2 = phibar * p2 + p2 * (pb2 - m) * inv_tau;
  // radial unit e = (x, y) / rho: ebar = pi0 (gbar_x, gbar_y)
  float ebx = p0 * gbar.x, eby = p0 * gbar.y;
  float ee = ex * ebx + ey * eby;
  float xb = (ebx - ex * ee) * irho + sb0 * ex;
  float yb = (eby - ey * ee) * irho + sb0 * ey;
  ybar += v3(xb, yb, sb1 - sb2);
  dbar += v3(-sb0, -sb1 - sb2, 0.f);
}

// Superquadric union (rows as in sdf_sq_union).  With pi_l = exp((phi - phi_l) / tau)
// and G_l = R_l grad_x f_l the forward has phi = -tau ln sum exp(-phi_l / tau) and
// g = sum_l pi_l G_l, so
//   phibar_l = pi_l (phibar - (gbar . G_l - gbar . g) / tau),
//   xbar_l   = phibar_l grad_x phi_l + H_l (pi_l R_l^T gbar),   ybar += R_l xbar_l,
// with grad_x phi_l = h f^(-h-1) |x| grad_x f + (1 - f^-h) x / |x| and H_l the
// Hessian of f_l:  d2f/dx~2 = r (r-1) s^(r-2) u'^2 + r s^(r-1) u'',
// d2f/dx~dy~ = r (r-1) s^(r-2) u' v', d2f/dz~2 = p1 (p1-1) |z~|^(p1-2), u' = p2
// |x~|^(p2-1) sgn x~, u'' = p2 (p2-1) |x~|^(p2-2), divided by the semi-axes of
// both indices.  As in the forward every power is an exp2 of a sum of base-2
// logarithms with log2 pi_l folded in.
CM_HD_OUTLINE void sdf_sq_union_bwd(V3 y, const float4* P, int L, const Sdf& f, float inv_tau, float phibar, V3 gbar,
                            V3& ybar) {
  const float k = inv_tau * kLog2e;
  const float gg = dot(gbar, f.g);
  V3 acc = v3(0.f, 0.f, 0.f);
  for (int l = 0; l < L; ++l) {
    const float4 r0 = P[5 * l], r1 = P[5 * l + 1], r2 = P[5 * l + 2], r3 = P[5 * l + 3], r4 = P[5 * l + 4];
    const V3 x = v3(fmaf(r0.x, y.x, fmaf(r0.y, y.y, fmaf(r0.z, y.z, r0.w))),
                    fmaf(r1.x, y.x, fmaf(r1.y, y.y, fmaf(r1.z, y.z, r1.w))),
                    fmaf(r2.x, y.x, fmaf(r2.y, y.y, fmaf(r2.z, y.z, r2.w))));
    const float xx = x.x * r3.x, xy = x.y * r3.y, xz = x.z * r3.z;
    const float p1 = r3.w, p2 = r4.x, rr = r4.y, h = r4.z;
    const float lx = lg2(fmaxf(fabsf(xx), 1e-20f)), ly = lg2(fmaxf(fabsf(xy), 1e-20f)),
                lz = lg2(fmaxf(fabsf(xz), 1e-20f));
    const float ls = log2_add(p2 * lx, p2 * ly);
    const float lf = log2_add(rr * ls, p1 * lz);
    const float fh = ex2(-h * lf);
    const float rho2 = dot(x, x);
    const float irho = rho2 > 0.f ? rsq(rho2) : 0.f;
    const float rho = rho2 * irho;
    const float le = (f.phi - (1.f - fh) * rho) * k;        // log2 pi_l
    const float pi = ex2(le);
    const V3 w = v3(dot(v3(r0.x, r0.y, r0.z), gbar), dot(v3(r1.x, r1.y, r1.z), gbar),
                    dot(v3(r2.x, r2.y, r2.z), gbar));     // R_l^T gbar
    const float Ex = (rr - 1.f) * ls + (p2 - 1.f) * lx, Ey = (rr - 1.f) * ls + (p2 - 1.f) * ly,
                Ez = (p1 - 1.f) * lz;
    const float cxy = rr * p2;
    // pi_l grad_x f
    const V3 gp = v3(copysignf(cxy * ex2(le + Ex), xx) * r3.x, copysignf(cxy * ex2(le + Ey), xy) * r3.y,
                     copysignf(p1 * ex2(le + Ez), xz) * r3.z);
    const float phib = pi * phibar - (dot(gp, w) - pi * gg) * inv_tau;
    // grad_x phi_l
    const float q = -(h + 1.f) * lf, hr = h * rho, om = (1.f - fh) * irho;
    const V3 dp = v3(fmaf(hr, copysignf(cxy * ex2(Ex + q), xx) * r3.x, om * x.x),
                     fmaf(hr, copysignf(cxy * ex2(Ey + q), xy) * r3.y, om * x.y),
                     fmaf(hr, copysignf(p1 * ex2(Ez + q), xz) * r3.z, om * x.z));
    V3 xb = dp * phib;
    // Hessian of f applied to pi_l R_l^T gbar
    const float T = le + (rr - 2.f) * ls;
    const float c2 = rr * (rr - 1.f) * p2 * p2, c1 = rr * p2 * (p2 - 1.f);
    const float Bx = (p2 - 1.f) * lx, By = (p2 - 1.f) * ly;
    const float hxx = c2 * ex2(T + 2.f * Bx) + c1 * ex2(le + (rr - 1.f) * ls + Bx - lx);
    const float hyy = c2 * ex2(T + 2.f * By) + c1 * ex2(le + (rr - 1.f) * ls + By - ly);
    const float hxy = copysignf(1.f, xx) * copysignf(1.f, xy) * c2 * ex2(T + Bx + By);
    const float hzz = p1 * (p1 - 1.f) * ex2(le + (p1 - 2.f) * lz);
    const float wx = w.x * r3.x, wy = w.y * r3.y, wz = w.z * r3.z;
    xb.x = fmaf(r3.x, fmaf(hxx, wx, hxy * wy), xb.x);
    xb.y = fmaf(r3.y, fmaf(hxy, wx, hyy * wy), xb.y);
    xb.z = fmaf(r3.z, hzz * wz, xb.z);
    acc.x += fmaf(xb.x, r0.x, fmaf(xb.y, r1.x, xb.z * r2.x));
    acc.y += fmaf(xb.x, r0.y, fmaf(xb.y, r1.y, xb.z * r2.y));
    acc.z += fmaf(xb.x, r0.z, fmaf(xb.y, r1.z, xb.z * r2.z));
  }
  ybar += acc;
}

CM_HD void body_sdf_bwd(const Body& b, V3 y, const Sdf& f, float tau, float inv_tau, float phibar, V3 gbar,
                        V3& ybar, V3& dbar) {
  switch (b.kind) {
    case kBox: sdf_box_bwd(y, b.dims, f, inv_tau, phibar, gbar, ybar, dbar); break;
    case kEllipsoid: sdf_ellipsoid_bwd(y, b.dims, phibar, gbar, ybar, dbar); break;
    case kCapsule: sdf_capsule_bwd(y, b.dims.x, b.dims.y, tau, inv_tau, phibar, gbar, ybar, dbar); break;
    case kCylinder: sdf_cylinder_bwd(y, b.dims.x, b.dims.y, f, inv_tau, phibar, gbar, ybar, dbar); break;
    case kSqUnion: sdf_sq_union_bwd(y, b.planes, b.n_planes / 5, f, inv_tau, phibar, gbar, ybar); break;
    default: sdf_planes_bwd(y, b.planes, b.n_planes, f, inv_tau, phibar, gbar, ybar); break;
  }
}

// A body's SDF at the two points an edge pair uses, with what the reverse needs
// (see sdf_planes2_h): value and gradient at y1 and at y2, and for a polyhedron
// the Hessian at y2.
struct Sdf2H {
  Sdf f1, f2;
  float H[6];
};
// The two evaluations of a primitive share one copy of its code (a loop that is
// not unrolled), which keeps the adjoint's edge-pair loop small in the
// instruction cache.
CM_HD Sdf2H body_sdf2_h(const Body& b, V3 y1, V3 y2, float tau, float inv_tau) {
  Sdf2H o;
  if (b.kind == kHull) {
    sdf_planes2_h(y1, y2, b.planes, b.n_planes, tau, o.f1, o.f2, o.H);
  } else {
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      const Sdf f = body_sdf(b, j ? y2 : y1, tau, inv_tau);
      if (j) o.f2 = f;
      else o.f1 = f;
    }
  }
  return o;
}
// Reverse of body_sdf2_h: phibar1 at y1, (phibar2, gbar2) at y2.  A polyhedron needs
// no pass over its planes: ybar1 += phibar1 g1, ybar2 += phibar2 g2 + H2 gbar2.
CM_HD void body_sdf2_h_bwd(const Body& b, V3 y1, V3 y2, const Sdf2H& s, float tau, float inv_tau, float phibar1,
                           float phibar2, V3 gbar2, V3& ybar1, V3& ybar2, V3& dbar) {
  if (b.kind == kHull) {
    const float* H = s.H;
    ybar1 += s.f1.g * phibar1;
    ybar2 += s.f2.g * phibar2 + v3(fmaf(H[0], gbar2.x, fmaf(H[1], gbar2.y, H[2] * gbar2.z)),
                                   fmaf(H[1], gbar2.x, fmaf(H[3], gbar2.y, H[4] * gbar2.z)),
                                   fmaf(H[2], gbar2.x, fmaf(H[4], gbar2.y, H[5] * gbar2.z)));
  } else {
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
      V3 yb = v3(0.f, 0.f, 0.f);
      body_sdf_bwd(b, j ? y2 : y1, j ? s.f2 : s.f1, tau, inv_tau, j ? phibar2 : phibar1,
                   j ? gbar2 : v3(0.f, 0.f, 0.f), yb, dbar);
      if (j) ybar2 += yb;
      else ybar1 += yb;
    }
  }
}

// Pair classes of the reverse: 0 any kinds; 1 A a polyhedron (hull) and B a box,
// capsule, cylinder or ellipsoid; 2 the other way round -- compiled without the kind
// dispatch and the branches the other kinds need.  kRole 0 is body A, 1 body B.
CM_HD constexpr bool is_hull_role(int kRole, int kCls) { return (kCls == 1 && kRole == 0) || (kCls == 2 && kRole == 1); }
CM_HD void prim_sdf_bwd(const Body& b, V3 y, const Sdf& f, float tau, float inv_tau, float phibar, V3 gbar,
                        V3& ybar, V3& dbar) {
  switch (b.kind) {
    case kBox: sdf_box_bwd(y, b.dims, f, inv_tau, phibar, gbar, ybar, dbar); break;
    case kEllipsoid: sdf_ellipsoid_bwd(y, b.dims, phibar, gbar, ybar, dbar); break;
    case kCapsule: sdf_capsule_bwd(y, b.dims.x, b.dims.y, tau, inv_tau, phibar, gbar, ybar, dbar); break;
    default: sdf_cylinder_bwd(y, b.dims.x, b.dims.y, f, inv_tau, phibar, gbar, ybar, dbar); break;
  }
}
// body_sdf2_h of body A (kRole 0) or B (kRole 1) in pair class kCls.  `plain`: the
// polyhedron's sums are taken without a shift (sdf_planes2_h_ee; y2 is the body's own
// witness within a scaled distance of 60 of its edge).
template <int kRole, int kCls>
CM_HD Sdf2H sdf2h_of(const Body& b, V3 y1, V3 y2, float tau, float inv_tau, bool plain = false) {
  if (kCls != 0) {
    Sdf2H o;
    if (is_hull_role(kRole, kCls)) {
      if (plain) sdf_planes2_h_ee(y1, y2, b.planes, b.n_planes, tau, o.f1, o.f2, o.H);
      else sdf_planes2_h(y1, y2, b.planes, b.n_planes, tau, o.f1, o.f2, o.H);
    } else {
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        const Sdf f = prim_sdf(b, j ? y2 : y1, tau, inv_tau);
        if (j) o.f2 = f;
        else o.f1 = f;
      }
    }
    return o;
  }
  return body_sdf2_h(b, y1, y2, tau, inv_tau);
}
template <int kRole, int kCls>
CM_HD void sdf2h_bwd_of(const Body& b, V3 y1, V3 y2, const Sdf2H& s, float tau, float inv_tau, float phibar1,
                        float phibar2, V3 gbar2, V3& ybar1, V3& ybar2, V3& dbar) {
  if (kCls != 0) {
    if (is_hull_role(kRole, kCls)) {
      const float* H = s.H;
      ybar1 += s.f1.g * phibar1;
      ybar2 += s.f2.g * phibar2 + v3(fmaf(H[0], gbar2.x, fmaf(H[1], gbar2.y, H[2] * gbar2.z)),
                                     fmaf(H[1], gbar2.x, fmaf(H[3], gbar2.y, H[4] * gbar2.z)),
                                     fmaf(H[2], gbar2.x, fmaf(H[4], gbar2.y, H[5] * gbar2.z)));
    } else {
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        V3 yb = v3(0.f, 0.f, 0.f);
        prim_sdf_bwd(b, j ? y2 : y1, j ? s.f2 : s.f1, tau, inv_tau, j ? phibar2 : phibar1,
                     j ? gbar2 : v3(0.f, 0.f, 0.f), yb, dbar);
        if (j) ybar2 += yb;
        else ybar1 += yb;
      }
    }
    return;
  }
  body_sdf2_h_bwd(b, y1, y2, s, tau, inv_tau, phibar1, phibar2, gbar2, ybar1, ybar2, dbar);
}

// One point of body_sdf2_h / body_sdf2_h_bwd.
struct Sdf1H {
  Sdf f;
  float H[6];
};
CM_HD Sdf1H body_sdf_h(const Body& b, V3 y, float tau, float inv_tau) {
  Sdf1H o;
  if (b.kind == kHull) sdf_planes_h(y, b.planes, b.n_planes, tau, o.f, o.H);
  else o.f = body_sdf(b, y, tau, inv_tau);
  return o;
}
CM_HD void body_sdf_h_bwd(const Body& b, V3 y, const Sdf1H& s, float tau, float inv_tau, float phibar, V3 gbar,
                          V3& ybar, V3& dbar) {
  if (b.kind == kHull) {
    const float* H = s.H;
    ybar += s.f.g * phibar + v3(fmaf(H[0], gbar.x, fmaf(H[1], gbar.y, H[2] * gbar.z)),
                                fmaf(H[1], gbar.x, fmaf(H[3], gbar.y, H[4] * gbar.z)),
                                fmaf(H[2], gbar.x, fmaf(H[4], gbar.y, H[5] * gbar.z)));
  } else {
    body_sdf_bwd(b, y, s.f, tau, inv_tau, phibar, gbar, ybar, dbar);
  }
}

// body_sdf_h / body_sdf_h_bwd of body A (kRole 0) or B (kRole 1) in pair class kCls.
template <int kRole, int kCls>
CM_HD Sdf1H sdf1h_of(const Body& b, V3 y, float tau, float inv_tau) {
  if (kCls != 0) {
    Sdf1H o;
    if (is_hull_role(kRole, kCls)) sdf_planes_h(y, b.planes, b.n_planes, tau, o.f, o.H);
    else o.f = prim_sdf(b, y, tau, inv_tau);
    return o;
  }
  return body_sdf_h(b, y, tau, inv_tau);
}
template <int kRole, int kCls>
CM_HD void sdf1h_bwd_of(const Body& b, V3 y, const Sdf1H& s, float tau, float inv_tau, float phibar, V3 gbar,
                        V3& ybar, V3& dbar) {
  if (kCls != 0) {
    if (is_hull_role(kRole, kCls)) {
      const float* H = s.H;
      ybar += s.f.g * phibar + v3(fmaf(H[0], gbar.x, fmaf(H[1], gbar.y, H[2] * gbar.z)),
                                  fmaf(H[1], gbar.x, fmaf(H[3], gbar.y, H[4] * gbar.z)),
                                  fmaf(H[2], gbar.x, fmaf(H[4], gbar.y, H[5] * gbar.z)));
    } else {
      prim_sdf_bwd(b, y, s.f, tau, inv_tau, phibar, gbar, ybar, dbar);
    }
    return;
  }
  body_sdf_h_bwd(b, y, s, tau, inv_tau, phibar, gbar, ybar, dbar);
}

// Adds a local-frame adjoint to a pre-selected item's export slot (shared memory).
CM_HD void export3(float* dst, V3 v) {
  if (dst) {
#if defined(__CUDA_ARCH__)
    atomicAdd(dst, v.x);
    atomicAdd(dst + 1, v.y);
    atomicAdd(dst + 2, v.z);
#else
    dst[0] += v.x;
    dst[1] += v.y;
    dst[2] += v.z;
#endif
  }
}

// Reverse of trace_to_surface from x0 (iters <= 8): xbar of the traced point ->
// xbar of x0; SDF parameter adjoints into dbar.  Step i maps x_i to
// x_i - phi(x_i) u, so xbar_i = xbar_(i+1) - grad phi(x_i) (u . xbar_(i+1)) and
// ubar += -phi(x_i) xbar_(i+1); u = g_0 / |g_0| hands (ubar - (ubar . u) u) / |g_0|
// to the gradient adjoint of the SDF at x0.
CM_HD_OUTLINE V3 trace_bwd(const Body& b, V3 x0, int iters, float tau, float it, V3 xbar, V3& dbar) {
  V3 xs[8];
  const Sdf s0 = body_sdf(b, x0, tau, it);
  const float ig = rsq(dot(s0.g, s0.g));
  const V3 u = s0.g * ig;
  V3 x = x0;
  for (int i = 0; i < iters; ++i) {
    xs[i] = x;
    x = fma3(-(i ? body_sdf(b, x, tau, it).phi : s0.phi), u, x);
  }
  V3 ub = v3(0.f, 0.f, 0.f);
  for (int i = iters - 1; i >= 0; --i) {
    const Sdf si = i ? body_sdf(b, xs[i], tau, it) : s0;
    const float phib = -dot(u, xbar);
    ub = fma3(-si.phi, xbar, ub);
    V3 gb = v3(0.f, 0.f, 0.f);
    if (i == 0) gb = (ub - u * dot(ub, u)) * ig;
    body_sdf_bwd(b, xs[i], si, tau, it, phib, gb, xbar, dbar);
  }
  return xbar;
}

// ---------------------------------------------------------------- vertex templates
// v = map(kind, u, dims) -> dims adjoint from the mapped vertex v and its cap sign s.
CM_HD void map_vertex_bwd(int kind, V3 v, float s, V3 d, V3 vbar, V3& dbar) {
  switch (kind) {
    case kBox:
    case kEllipsoid:
      dbar += v3(vbar.x * v.x * rcp(d.x), vbar.y * v.y * rcp(d.y), vbar.z * v.z * rcp(d.z));
      break;
    case kCylinder:
      dbar += v3((vbar.x * v.x + vbar.y * v.y) * rcp(d.x), vbar.z * v.z * rcp(d.y), 0.f);
      break;
    case kCapsule: {
      float ir = rcp(d.x);
      V3 u = v3(v.x * ir, v.y * ir, (v.z - s * d.y) * ir);
      dbar += v3(dot(vbar, u), vbar.z * s, 0.f);
      break;
    }
    default: break;
  }
}

// ---------------------------------------------------------------- E-E box QP
// Reverse of qp_setup + qp_solve: (abar1, abar2, conbar) -> adjoints of a0, a1, b0, b1.
CM_HD void qp_bwd(const QPPre& q, float lam, const Params& p, float ab1, float ab2, float conb, V3& a0b, V3& a1b,
                  V3& b0b, V3& b1b) {
  // ---- forward recompute
  V3 X = cross(q.t1, q.t2);
  float T11 = q.Q11 - lam, T22 = q.Q22 - lam, T12 = q.Q12;
  float B1 = q.c1 + 0.5f * lam, B2 = q.c2 + 0.5f * lam;
  float det = dot(X, X) + lam * (T11 + T22) + lam * lam;
  float n1 = -dot(X, cross(q.b, q.t2)) + lam * (0.5f * (T22 - T12) - B1 + 0.5f * lam);
  float n2 = -dot(X, cross(q.t1, q.b)) + lam * (0.5f * (T11 - T12) - B2 + 0.5f * lam);
  float idet = rcp(det);
  float au1 = n1 * idet, au2 = n2 * idet;
  float ie = rcp(p.eps_clip);
  float iQ11 = rcp(q.Q11), iQ22 = rcp(q.Q22);
  float z1 = -(q.Q12 + q.c2) * iQ22, z2 = -q.c2 * iQ22, z3 = -(q.Q12 + q.c1) * iQ11, z4 = -q.c1 * iQ11;
  // the soft clips with their derivatives (sharing each side's exponentials)
  float cg1, cg2, cg3, cg4;
  float s1 = clip01_s_vg(z1, ie, p.eps_clip, cg1), s2 = clip01_s_vg(z2, ie, p.eps_clip, cg2);
  float s3 = clip01_s_vg(z3, ie, p.eps_clip, cg3), s4 = clip01_s_vg(z4, ie, p.eps_clip, cg4);
  float J1 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, 1.f, s1);
  float J2 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, 0.f, s2);
  float J3 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, s3, 1.f);
  float J4 = qp_cost(q.Q11, q.Q12, q.Q22, q.c1, q.c2, s4, 0.f);
  float Jm = fminf(fminf(J1, J2), fminf(J3, J4));
  float iem = rcp(p.eps_min);
  float k = -iem * kLog2e;
  float w1 = ex2((J1 - Jm) * k), w2 = ex2((J2 - Jm) * k), w3 = ex2((J3 - Jm) * k), w4 = ex2((J4 - Jm) * k);
  float iw = rcp((w1 + w2) + (w3 + w4));
  float pr1 = w1 * iw, pr2 = w2 * iw, pr3 = w3 * iw, pr4 = w4 * iw;
  float ac1 = pr1 + pr3 * s3 + pr4 * s4;
  float ac2 = pr1 * s1 + pr2 * s2 + pr3;
  float ic = rcp(p.eps_comp);
  float wg1, wg2;
  float wi1 = within01_vg(au1, ic, wg1), wi2 = within01_vg(au2, ic, wg2);
  float con = wi1 * wi2;

  // ---- reverse of alpha = con au + (1 - con) ac
  float aub1 = con * ab1, aub2 = con * ab2;
  float acb1 = (1.f - con) * ab1, acb2 = (1.f - con) * ab2;
  float cb = conb + ab1 * (au1 - ac1) + ab2 * (au2 - ac2);
  aub1 += cb * wi2 * wg1;
  aub2 += cb * wi1 * wg2;

  // ---- soft argmin: ac = sum_j pr_j a_j, candidates (1, s1), (0, s2), (s3, 1), (s4, 0)
  float pb1 = acb1 + acb2 * s1, pb2 = acb2 * s2, pb3 = acb1 * s3 + acb2, pb4 = acb1 * s4;
  float sbar1 = pr1 * acb2, sbar2 = pr2 * acb2, sbar3 = pr3 * acb1, sbar4 = pr4 * acb1;
  float pm = pr1 * pb1 + pr2 * pb2 + pr3 * pb3 + pr4 * pb4;
  float Jb1 = -iem * pr1 * (pb1 - pm), Jb2 = -iem * pr2 * (pb2 - pm), Jb3 = -iem * pr3 * (pb3 - pm),
        Jb4 = -iem * pr4 * (pb4 - pm);

  // ---- costs J(a) = 1/2 a^T Q a + c^T a
  float Qb11 = 0.f, Qb12 = 0.f, Qb22 = 0.f, cb1 = 0.f, cb2 = 0.f;
  auto cost_bwd = [&](float Jb, float x1, float x2, float& x1b, float& x2b) {
    Qb11 += Jb * 0.5f * x1 * x1;
    Qb12 += Jb * x1 * x2;
    Qb22 += Jb * 0.5f * x2 * x2;
    cb1 += Jb * x1;
    cb2 += Jb * x2;
    x1b += Jb * (q.Q11 * x1 + q.Q12 * x2 + q.c1);
    x2b += Jb * (q.Q12 * x1 + q.Q22 * x2 + q.c2);
  };
  float dummy = 0.f;
  cost_bwd(Jb1, 1.f, s1, dummy, sbar1);
  cost_bwd(Jb2, 0.f, s2, dummy, sbar2);
  cost_bwd(Jb3, s3, 1.f, sbar3, dummy);
  cost_bwd(Jb4, s4, 0.f, sbar4, dummy);

  // ---- side minimisers z_j through the soft clip
  float zb1 = sbar1 * cg1, zb2 = sbar2 * cg2;
  float zb3 = sbar3 * cg3, zb4 = sbar4 * cg4;
  // z1 = -(Q12 + c2)/Q22, z2 = -c2/Q22, z3 = -(Q12 + c1)/Q11, z4 = -c1/Q11
  Qb12 += -zb1 * iQ22 - zb3 * iQ11;
  cb2 += -(zb1 + zb2) * iQ22;
  cb1 += -(zb3 + zb4) * iQ11;
  Qb22 += -(zb1 * z1 + zb2 * z2) * iQ22;
  Qb11 += -(zb3 * z3 + zb4 * z4) * iQ11;

  // ---- unconstrained minimiser au = -Q^-1 c:  cbar = -v, Qbar = -v au^T with v = Q^-1 aubar
  float v1 = (q.Q22 * aub1 - q.Q12 * aub2) * idet;
  float v2 = (-q.Q12 * aub1 + q.Q11 * aub2) * idet;
  cb1 -= v1;
  cb2 -= v2;
  Qb11 -= v1 * au1;
  Qb22 -= v2 * au2;
  Qb12 -= v1 * au2 + v2 * au1;

  // ---- Q = A^T A + lam I, c = A^T b - lam/2 with A = [t1, t2]
  V3 t1b = q.t1 * (2.f * Qb11) + q.t2 * Qb12 + q.b * cb1;
  V3 t2b = q.t2 * (2.f * Qb22) + q.t1 * Qb12 + q.b * cb2;
  V3 bb = q.t1 * cb1 + q.t2 * cb2;
  // t1 = a1 - a0, t2 = b0 - b1, b = a0 - b0
  a1b += t1b;
  a0b += bb - t1b;
  b0b += t2b - bb;
  b1b += -t2b;
}

// ---------------------------------------------------------------- frame of a pair
// Everything is evaluated in B's frame; A-local x maps to R_rel x + t_rel.
struct Frame {
  M3 R;
  V3 t;
  float tau, inv_tau, k2;
};

// A-local point x with adjoint xbar at B-frame point y = R x + t  (x = R^T (y - t)).
CM_HD V3 pull_point_bwd(const Frame& F, V3 y, V3 xbar, Adj& adj) {
  V3 Rx = mul(F.R, xbar);
  adj.t += -Rx;
  add_outer(adj.R, y - F.t, xbar);
  return Rx;  // ybar contribution
}
// B-frame point y = R v + t of an A-local vertex v: ybar -> (adj.R, adj.t), returns vbar (local).
CM_HD V3 push_point_bwd(const Frame& F, V3 v, V3 ybar, Adj& adj) {
  add_outer(adj.R, ybar, v);
  adj.t += ybar;
  return mulT(F.R, ybar);
}

// ---------------------------------------------------------------- vertex-SDF candidate
// Candidate of A's vertex (vL local, vB in B's frame) against B, or of B's
// vertex (vB) against A.  Upstream: yb[8] for (p, d, n, w) in B's frame, sb for
// the score s = -w d.
template <bool kOfA, int kCls = 0>
CM_HD void vs_bwd(const Frame& F, const Body& A, const Body& B, float4 vL, V3 vB, const float (&yb)[8], float sb,
                  Adj& adj, float* vexp = nullptr) {
  const float tau = F.tau, it = F.inv_tau;
  if (kOfA) {
    const Sdf1H fh = sdf1h_of<1, kCls>(B, vB, tau, it);
    const Sdf& f = fh.f;
    float w = sigmoid(-f.phi * it);
    float wb = yb[7] - sb * f.phi;
    float phib = yb[3] - sb * w - wb * sigmoid_grad_from(w) * it;
    V3 gb = normal_bwd(f.g, tau, v3(yb[4], yb[5], yb[6]));
    V3 pb = v3(yb[0], yb[1], yb[2]);
    sdf1h_bwd_of<1, kCls>(B, vB, fh, tau, it, phib, gb, pb, adj.dB);
    V3 vl = v3(vL.x, vL.y, vL.z);
    V3 vbar = push_point_bwd(F, vl, pb, adj);
    if (!is_hull_role(0, kCls)) map_vertex_bwd(A.kind, vl, vL.w, A.dims, vbar, adj.dA);
    export3(vexp, vbar);
  } else {
    V3 x = mulT(F.R, vB - F.t);
    const Sdf1H fh = sdf1h_of<0, kCls>(A, x, tau, it);
    const Sdf& f = fh.f;
    float w = sigmoid(-f.phi * it);
    float wb = yb[7] - sb * f.phi;
    float phib = yb[3] - sb * w - wb * sigmoid_grad_from(w) * it;
    V3 nub = v3(yb[4], yb[5], yb[6]);            // n = R nu_local
    V3 nuL = normal_of(f.g, tau);
    add_outer(adj.R, nub, nuL);
    V3 gb = normal_bwd(f.g, tau, mulT(F.R, nub));
    V3 xb = v3(0.f, 0.f, 0.f);
    sdf1h_bwd_of<0, kCls>(A, x, fh, tau, it, phib, gb, xb, adj.dA);
    V3 pb = v3(yb[0], yb[1], yb[2]) + pull_point_bwd(F, vB, xb, adj);
    map_vertex_bwd(B.kind, vB, vL.w, B.dims, pb, adj.dB);
    export3(vexp, pb);
  }
}

// ---------------------------------------------------------------- witness + QP reverse
struct EEGeom {
  float4 a0, a1;    // A's edge in B's frame (w unused)
  float4 a0L, a1L;  // A's edge in A's frame (w = capsule cap sign)
  float4 b0, b1;    // B's edge (w = capsule cap sign)
};
CM_HD V3 xyz(float4 f) { return v3(f.x, f.y, f.z); }

// Endpoint adjoints -> relative pose, dims of both bodies and the pre-selected edges'
// exports: a0b, a1b for A's endpoints in B's frame, l0x, l1x added to them in A's
// own frame, b0b, b1b for B's.
template <int kCls = 0>
CM_HD void endpoints_bwd(const Frame& F, const Body& A, const Body& B, const EEGeom& g, V3 a0b, V3 a1b, V3 l0x,
                         V3 l1x, V3 b0b, V3 b1b, Adj& adj, float* eAexp, float* eBexp) {
  const V3 a0L = xyz(g.a0L), a1L = xyz(g.a1L), b0 = xyz(g.b0), b1 = xyz(g.b1);
  const V3 l0 = push_point_bwd(F, a0L, a0b, adj) + l0x;
  const V3 l1 = push_point_bwd(F, a1L, a1b, adj) + l1x;
  if (!is_hull_role(0, kCls)) {  // a hull's vertices are fixed: no dims to map
    map_vertex_bwd(A.kind, a0L, g.a0L.w, A.dims, l0, adj.dA);
    map_vertex_bwd(A.kind, a1L, g.a1L.w, A.dims, l1, adj.dA);
  }
  if (!is_hull_role(1, kCls)) {
    map_vertex_bwd(B.kind, b0, g.b0.w, B.dims, b0b, adj.dB);
    map_vertex_bwd(B.kind, b1, g.b1.w, B.dims, b1b, adj.dB);
  }
  // pre-selected edges: their endpoints' local adjoints feed the selection's reverse
  if (eAexp) {
    export3(eAexp, l0);
    export3(eAexp + 3, l1);
  }
  if (eBexp) {
    export3(eBexp, b0b);
    export3(eBexp + 3, b1b);
  }
}

// Witness reverse at a fixed QP result: e1 = a0 + al1 (a1 - a0) in B's frame (e1L
// likewise in A's frame), e2 = b0 + al2 (b1 - b0).  The endpoints' adjoints at fixed
// alpha go to the parameters; the alpha adjoints are returned for the QP's reverse.
template <int kCls = 0>
CM_HD void witness_direct_bwd(const Frame& F, const Body& A, const Body& B, const EEGeom& g, const QPOut& o, V3 e1b,
                              V3 e1Lb, V3 e2b, Adj& adj, float& ab1, float& ab2, float* eAexp, float* eBexp) {
  const V3 a0 = xyz(g.a0), a1 = xyz(g.a1), b0 = xyz(g.b0), b1 = xyz(g.b1);
  ab1 = dot(e1b, a1 - a0) + dot(e1Lb, xyz(g.a1L) - xyz(g.a0L));
  ab2 = dot(e2b, b1 - b0);
  endpoints_bwd<kCls>(F, A, B, g, e1b * (1.f - o.a1), e1b * o.a1, e1Lb * (1.f - o.a1), e1Lb * o.a1, e2b * (1.f - o.a2),
                e2b * o.a2, adj, eAexp, eBexp);
}

// The adjoints of an edge pair's QP result (alpha1, alpha2, con), summed over every use.
struct QPBar {
  float a1, a2, con;
};

// ---------------------------------------------------------------- E-E element
// Recomputes both candidates of an edge pair, asks `up` for their upstream
// adjoints, and backpropagates them to the witness points and from there, at the
// fixed QP result, to the parameters.  Two parts are left to the caller's last
// pass over the edge pairs: the nearest-neighbour softmax's dependence on the
// distance matrix, returned as t_b = nnbar_b * nn_b, and the QP's own reverse,
// whose (alpha, con) adjoints are returned, so that it runs once per edge pair
// with the distance adjoint's share added.
struct EECand {
  float y1[8], y2[8];
  float s1, s2;
};

// The SDFs come from sdf2h_of (a polyhedron's value, gradient and Hessian in one pass
// over its planes), so their reverses need no second pass; kCls is the pair class (see
// sdf2h_of).  dqp (optional) receives the QP witnesses' distance.
template <int kCls = 0, class Upstream>
CM_HD QPBar ee_bwd(const Frame& F, const Body& A, const Body& B, const Params& p, const EEGeom& g, float rowL,
                  float colL, const QPOut* stored, Upstream&& up, float& t1, float& t2, Adj& adj,
                  float* eAexp = nullptr, float* eBexp = nullptr, float* dqp = nullptr) {
  const float tau = F.tau, it = F.inv_tau;
  V3 a0 = xyz(g.a0), a1 = xyz(g.a1), b0 = xyz(g.b0), b1 = xyz(g.b1);
  V3 a0L = xyz(g.a0L), a1L = xyz(g.a1L);
  // ---- forward recompute (the QP result may come from the pass that built the distances)
  QPPre q = qp_setup(a0, a1, b0, b1, p.w_reg);
  QPOut o = stored ? *stored : qp_solve(q, p.w_reg, p);
  V3 e1 = fma3(o.a1, a1 - a0, a0), e2 = fma3(o.a2, b1 - b0, b0);
  V3 e1L = fma3(o.a1, a1L - a0L, a0L);
  // nn indicators rank the QP witnesses' distances; sphere tracing (if on) moves
  // the witnesses everything else uses
  const float dbar_qp = sqrt_(dot(e1 - e2, e1 - e2));
  if (dqp) *dqp = dbar_qp;
  const int nt = p.trace_iters;
  const V3 e1Lq = e1L, e2q = e2;
  if (nt) {
    e1L = trace_to_surface(A, e1L, nt, tau, it);
    e2 = trace_to_surface(B, e2, nt, tau, it);
    e1 = mul(F.R, e1L) + F.t;
  }
  V3 D = e1 - e2;
  float r2 = dot(D, D);
  float dbar = sqrt_(r2);
  float qn = rsq(r2 + tau * tau);
  V3 nbar = D * qn;
  V3 x2 = mulT(F.R, e2 - F.t);
  // the polyhedron of the pair class sums its planes without a shift while its own
  // witness (at alpha on its edge's line, no sphere tracing, no soft pre-selection) is
  // within a scaled distance of 60 of the edge, as the forward does
  const bool guard = p.top_verts > 0 || p.top_edges > 0;
  bool plain = false;
  if (kCls != 0 && !nt && !guard) {
    const float al = kCls == 1 ? o.a1 : o.a2;
    const V3 te = kCls == 1 ? a1L - a0L : b1 - b0;
    const float ex = fmaxf(fmaxf(-al, al - 1.f), 0.f) * F.k2;
    plain = ex * ex * dot(te, te) <= 3600.f;
  }
  const Sdf2H hB = sdf2h_of<1, kCls>(B, e1, e2, tau, it, plain);   // phi_B(e1*), nu_B(e2*)
  const Sdf2H hA = sdf2h_of<0, kCls>(A, x2, e1L, tau, it, plain);  // phi_A(e2*), nu_A(e1*) in A's frame
  const Sdf &SB1 = hB.f1, &SB2 = hB.f2, &SA2 = hA.f1, &SA1 = hA.f2;
  V3 nuB = normal_of(SB2.g, tau);
  V3 nuAL = normal_of(SA1.g, tau);
  V3 nuA = mul(F.R, nuAL);
  float g1 = tanh_(dot(nuB, nbar) * it), g2 = tanh_(-dot(nuA, nbar) * it);
  float pen1 = sigmoid(-SB1.phi * it), pen2 = sigmoid(-SA2.phi * it);
  float cl = sigmoid(-dot(nuA, nuB) * it);
  float nn1 = ex2((rowL - dbar_qp) * F.k2), nn2 = ex2((colL - dbar_qp) * F.k2);
  float con = o.con;
  // pre-selection's safeguard (Supplement B): each witness inside its own body
  const float sg1 = guard ? sigmoid(-SA1.phi * it) : 1.f, sg2 = guard ? sigmoid(-SB2.phi * it) : 1.f;
  const float pr1 = pen1, pr2 = pen2;  // the penetration indicators without the safeguard
  pen1 *= sg1;
  pen2 *= sg2;
  float w1 = con * cl * pen1 * nn1, w2 = con * cl * pen2 * nn2;
  EECand c;
  c.y1[0] = e1.x; c.y1[1] = e1.y; c.y1[2] = e1.z; c.y1[3] = g1 * dbar;
  c.y1[4] = g1 * nbar.x; c.y1[5] = g1 * nbar.y; c.y1[6] = g1 * nbar.z; c.y1[7] = w1;
  c.y2[0] = e2.x; c.y2[1] = e2.y; c.y2[2] = e2.z; c.y2[3] = g2 * dbar;
  c.y2[4] = -g2 * nbar.x; c.y2[5] = -g2 * nbar.y; c.y2[6] = -g2 * nbar.z; c.y2[7] = w2;
  c.s1 = -w1 * c.y1[3];
  c.s2 = -w2 * c.y2[3];
  float yb1[8], yb2[8], sb1, sb2;
  up(c, yb1, sb1, yb2, sb2);
  // ---- reverse
  float wb1 = yb1[7] - sb1 * c.y1[3], wb2 = yb2[7] - sb2 * c.y2[3];
  float db1 = yb1[3] - sb1 * w1, db2 = yb2[3] - sb2 * w2;
  V3 nb1 = v3(yb1[4], yb1[5], yb1[6]), nb2 = v3(yb2[4], yb2[5], yb2[6]);
  float gb1 = db1 * dbar + dot(nb1, nbar);
  float gb2 = db2 * dbar - dot(nb2, nbar);
  float dbarb = db1 * g1 + db2 * g2;
  V3 nbarb = nb1 * g1 - nb2 * g2;
  float conb = wb1 * cl * pen1 * nn1 + wb2 * cl * pen2 * nn2;
  float clb = wb1 * con * pen1 * nn1 + wb2 * con * pen2 * nn2;
  float penb1 = wb1 * con * cl * nn1, penb2 = wb2 * con * cl * nn2;
  t1 = wb1 * con * cl * pen1 * nn1;
  t2 = wb2 * con * cl * pen2 * nn2;
  // pen_b here includes the safeguard factor: split the adjoint between the two
  float phibB1 = -penb1 * sg1 * sigmoid_grad_from(pr1) * it;
  float phibA2 = -penb2 * sg2 * sigmoid_grad_from(pr2) * it;
  const float phibA1 = guard ? -penb1 * pr1 * sigmoid_grad_from(sg1) * it : 0.f;
  const float phibB2 = guard ? -penb2 * pr2 * sigmoid_grad_from(sg2) * it : 0.f;
  float cclb = -clb * sigmoid_grad_from(cl) * it;
  V3 nuAb = nuB * cclb, nuBb = nuA * cclb;
  float xb1 = gb1 * (1.f - g1 * g1) * it;
  float xb2 = gb2 * (1.f - g2 * g2) * it;
  nuBb += nbar * xb1;
  nbarb += nuB * xb1;
  nuAb += nbar * (-xb2);
  nbarb += nuA * (-xb2);
  V3 Db = nbarb * qn - D * (dot(D, nbarb) * qn * qn * qn);
  if (dbar > 0.f) Db += D * (dbarb * rcp(dbar));
  V3 e1b = Db + v3(yb1[0], yb1[1], yb1[2]);
  V3 e2b = -Db + v3(yb2[0], yb2[1], yb2[2]);
  // SDF reverses (one pass per body for its two points)
  sdf2h_bwd_of<1, kCls>(B, e1, e2, hB, tau, it, phibB1, phibB2, normal_bwd(SB2.g, tau, nuBb), e1b, e2b, adj.dB);
  V3 x2b = v3(0.f, 0.f, 0.f), e1Lb = v3(0.f, 0.f, 0.f);
  add_outer(adj.R, nuAb, nuAL);
  sdf2h_bwd_of<0, kCls>(A, x2, e1L, hA, tau, it, phibA2, phibA1, normal_bwd(SA1.g, tau, mulT(F.R, nuAb)), x2b, e1Lb,
                        adj.dA);
  e2b += pull_point_bwd(F, e2, x2b, adj);
  if (nt) {  // traced e1 = R_rel e1L + t_rel; back through both traces to the QP witnesses
    e1Lb += push_point_bwd(F, e1L, e1b, adj);
    e1Lb = trace_bwd(A, e1Lq, nt, tau, it, e1Lb, adj.dA);
    e2b = trace_bwd(B, e2q, nt, tau, it, e2b, adj.dB);
    e1b = v3(0.f, 0.f, 0.f);
  }
  QPBar qb;
  witness_direct_bwd<kCls>(F, A, B, g, o, e1b, e1Lb, e2b, adj, qb.a1, qb.a2, eAexp, eBexp);
  qb.con = conb;
  return qb;
}

// Last pass of an edge pair: the distance-matrix adjoint Dbar flows through
// dbar = |e1* - e2*| of the QP witnesses (its direct part to the endpoints, its alpha
// part added to the candidates' alpha adjoints), then the QP's reverse runs once on
// the total.
template <int kCls = 0>
CM_HD void ee_qp_bwd(const Frame& F, const Body& A, const Body& B, const Params& p, const EEGeom& g, float Dbar,
                     const QPOut& o, QPBar qb, Adj& adj, float* eAexp = nullptr, float* eBexp = nullptr) {
  const V3 a0 = xyz(g.a0), a1 = xyz(g.a1), b0 = xyz(g.b0), b1 = xyz(g.b1);
  const V3 z = v3(0.f, 0.f, 0.f);
  V3 a0b = z, a1b = z, b0b = z, b1b = z;  // endpoint adjoints of both parts, reversed to the parameters once
  bool any = false;
  if (Dbar != 0.f) {
    const V3 D = fma3(o.a1, a1 - a0, a0) - fma3(o.a2, b1 - b0, b0);
    const float r2 = dot(D, D);
    if (r2 > 0.f) {  // |e1* - e2*| at fixed alpha, and its alpha part
      const V3 Db = D * (Dbar * rsq(r2));
      a0b = Db * (1.f - o.a1);
      a1b = Db * o.a1;
      b0b = Db * (o.a2 - 1.f);
      b1b = Db * (-o.a2);
      qb.a1 += dot(Db, a1 - a0);
      qb.a2 -= dot(Db, b1 - b0);
      any = true;
    }
  }
  if (qb.a1 != 0.f || qb.a2 != 0.f || qb.con != 0.f) {
    const QPPre q = qp_setup(a0, a1, b0, b1, p.w_reg);
    qp_bwd(q, p.w_reg, p, qb.a1, qb.a2, qb.con, a0b, a1b, b0b, b1b);
    any = true;
  }
  if (any) endpoints_bwd<kCls>(F, A, B, g, a0b, a1b, z, z, b0b, b1b, adj, eAexp, eBexp);
}

// ---------------------------------------------------------------- pose epilogue
// R(q / |q|) reverse: Rbar (row-major) -> qbar for the raw quaternion (w, x, y, z).
CM_HD void quat_rot_bwd(const float* q4, const float* Rb, float* qb) {
  float n = sqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
  float in = 1.f / n;
  float w = q4[0] * in, x = q4[1] * in, y = q4[2] * in, z = q4[3] * in;
  const float* R = Rb;
  float gw = 2.f * (-z * R[1] + y * R[2] + z * R[3] - x * R[5] - y * R[6] + x * R[7]);
  float gx = 2.f * (y * R[1] + z * R[2] + y * R[3] - 2.f * x * R[4] - w * R[5] + z * R[6] + w * R[7] - 2.f * x * R[8]);
  float gy = 2.f * (-2.f * y * R[0] + x * R[1] + w * R[2] + x * R[3] + z * R[5] - w * R[6] + z * R[7] - 2.f * y * R[8]);
  float gz = 2.f * (-2.f * z * R[0] - w * R[1] + x * R[2] + w * R[3] - 2.f * z * R[4] + y * R[5] + x * R[6] + y * R[7]);
  float dp = gw * w + gx * x + gy * y + gz * z;
  qb[0] = (gw - w * dp) * in;
  qb[1] = (gx - x * dp) * in;
  qb[2] = (gy - y * dp) * in;
  qb[3] = (gz - z * dp) * in;
}

// Pair epilogue: adjoints of (R_rel, t_rel) plus the output-transform adjoints
// (Rb_out for R_B, tb_out for t_B) -> gradients of both poses (14 floats).
// R_rel = R_B^T R_A, t_rel = R_B^T (t_A - t_B).
CM_HD void pose_epilogue(const float* P, const M3& RA, const M3& RB, const Adj& adj, const float* Rb_out,
                         V3 tb_out, float* gpose) {
  float RAb[9], RBb[9];
  for (int i = 0; i < 9; ++i) RBb[i] = Rb_out[i];
  // R_rel = R_B^T R_A: RAb = R_B adj.R; RBb += R_A adj.R^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      float a = 0.f, b = 0.f;
      for (int k = 0; k < 3; ++k) {
        a += RB.m[i * 3 + k] * adj.R[k * 3 + j];
        b += RA.m[i * 3 + k] * adj.R[j * 3 + k];
      }
      RAb[i * 3 + j] = a;
      RBb[i * 3 + j] += b;
    }
  // t_rel = R_B^T (t_A - t_B)
  V3 d = v3(P[4] - P[11], P[5] - P[12], P[6] - P[13]);
  V3 tA_b = mul(RB, adj.t);
  add_outer(RBb, d, adj.t);
  quat_rot_bwd(P, RAb, gpose);
  gpose[4] = tA_b.x; gpose[5] = tA_b.y; gpose[6] = tA_b.z;
  quat_rot_bwd(P + 7, RBb, gpose + 7);
  gpose[11] = tb_out.x - tA_b.x; gpose[12] = tb_out.y - tA_b.y; gpose[13] = tb_out.z - tA_b.z;
}

}  // namespace cm
