// Host build of the adjoint's E-E element (ee_bwd: both candidates of an edge
// pair recomputed and reversed; ee_qp_bwd: the QP's reverse; pose_epilogue: the
// chain to the quaternion and translation) for tests/test_host_ee_element.py, on the
// kernels' two specialised pair classes -- class 1: A a convex polyhedron, B a box;
// class 2: A a box, B a convex polyhedron -- with one edge each, so that both
// nearest-neighbour indicators are 1.  Input: "tau F cls", F plane rows (n_x n_y n_z c
// in the polyhedron's frame, unnormalised by tau), then per line: qA(4) tA(3) a0(3)
// a1(3) b0(3) b1(3) h(3) yb1(8) sb1 yb2(8) sb2, where the edges are in their own
// body's frame (a box edge as template rows, scaled by the box's half-extents h) and
// yb, sb are the upstream adjoints of both candidates' rows (p, d, n, w) and scores
// s = -w d; B sits at the origin unrotated.  Output per line: y1(8) s1 y2(8) s2, the
// gradient of yb1 . y1 + sb1 s1 + yb2 . y2 + sb2 s2 with respect to qA(4), tA(3) and
// h(3), and 1 if the polyhedron's plain sums were taken (its witness within a scaled
// distance of 60 of its edge), else 0.
#include <cstdio>
#include <vector>

#include "cm_adjoint.cuh"

using namespace cm;

// Hands the element the given upstream adjoints and keeps its recomputed candidates.
struct Upstream {
  const float* v;
  EECand* cand;
  CM_HD void operator()(const EECand& c, float (&yb1)[8], float& sb1, float (&yb2)[8], float& sb2) const {
    *cand = c;
    for (int i = 0; i < 8; ++i) {
      yb1[i] = v[22 + i];
      yb2[i] = v[31 + i];
    }
    sb1 = v[30];
    sb2 = v[39];
  }
};

int main() {
  float tau;
  int F, cls;
  if (std::scanf("%f %d %d", &tau, &F, &cls) != 3 || F <= 0 || (cls != 1 && cls != 2)) return 2;
  const float k2 = kLog2e / tau;
  std::vector<float4> P(F);
  for (int f = 0; f < F; ++f) {
    float x, y, z, c;
    if (std::scanf("%f %f %f %f", &x, &y, &z, &c) != 4) return 2;
    P[f] = make_float4(k2 * x, k2 * y, k2 * z, k2 * c);  // staged as base-2 exponents
  }
  Params p{};
  p.tau = tau;
  p.w_reg = 0.01f;
  p.eps_clip = p.eps_min = p.eps_comp = 0.1f;
  p.K = 8;
  float v[40];
  for (;;) {
    int got = 0;
    for (int i = 0; i < 40; ++i) got += std::scanf("%f", &v[i]);
    if (got != 40) break;
    const float pose[14] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Frame Fr;
    Fr.R = quat_rot(v[0], v[1], v[2], v[3]);  // R_rel = R_A with B at the origin
    Fr.t = v3(v[4], v[5], v[6]);
    Fr.tau = tau;
    Fr.inv_tau = 1.f / tau;
    Fr.k2 = k2;
    const V3 h = v3(v[19], v[20], v[21]);
    const Body hull{kHull, v3(1.f, 1.f, 1.f), P.data(), F};
    const Body box{kBox, h, nullptr, 0};
    const Body& A = cls == 1 ? hull : box;
    const Body& B = cls == 1 ? box : hull;
    const V3 sa = cls == 1 ? v3(1.f, 1.f, 1.f) : h, sb = cls == 1 ? h : v3(1.f, 1.f, 1.f);
    const V3 a0L = v3(v[7] * sa.x, v[8] * sa.y, v[9] * sa.z), a1L = v3(v[10] * sa.x, v[11] * sa.y, v[12] * sa.z);
    const V3 b0 = v3(v[13] * sb.x, v[14] * sb.y, v[15] * sb.z), b1 = v3(v[16] * sb.x, v[17] * sb.y, v[18] * sb.z);
    const V3 a0 = mul(Fr.R, a0L) + Fr.t, a1 = mul(Fr.R, a1L) + Fr.t;
    EEGeom g;
    g.a0 = make_float4(a0.x, a0.y, a0.z, 0.f);
    g.a1 = make_float4(a1.x, a1.y, a1.z, 0.f);
    g.a0L = make_float4(a0L.x, a0L.y, a0L.z, 0.f);
    g.a1L = make_float4(a1L.x, a1L.y, a1L.z, 0.f);
    g.b0 = make_float4(b0.x, b0.y, b0.z, 0.f);
    g.b1 = make_float4(b1.x, b1.y, b1.z, 0.f);
    const QPOut o = qp_solve(qp_setup(a0, a1, b0, b1, p.w_reg), p.w_reg, p);
    // the QP witnesses' distance first, then the element with both row and column
    // minima equal to it (one edge per body: both nearest-neighbour indicators are 1)
    float dqp = 0.f, t1, t2;
    Adj adj;
    adj_zero(adj);
    EECand cand;
    Upstream up{v, &cand};
    QPBar qb;
    if (cls == 1) {
      ee_bwd<1>(Fr, A, B, p, g, 0.f, 0.f, &o, up, t1, t2, adj, nullptr, nullptr, &dqp);
      adj_zero(adj);
      qb = ee_bwd<1>(Fr, A, B, p, g, dqp, dqp, &o, up, t1, t2, adj);
      // distance-matrix adjoint of a 1 x 1 matrix: (nn1 R - t1 + nn2 C - t2) / tau = 0
      ee_qp_bwd<1>(Fr, A, B, p, g, ((t1 - t1) + (t2 - t2)) * Fr.inv_tau, o, qb, adj);
    } else {
      ee_bwd<2>(Fr, A, B, p, g, 0.f, 0.f, &o, up, t1, t2, adj, nullptr, nullptr, &dqp);
      adj_zero(adj);
      qb = ee_bwd<2>(Fr, A, B, p, g, dqp, dqp, &o, up, t1, t2, adj);
      ee_qp_bwd<2>(Fr, A, B, p, g, ((t1 - t1) + (t2 - t2)) * Fr.inv_tau, o, qb, adj);
    }
    const M3 RB = quat_rot(1.f, 0.f, 0.f, 0.f);
    const float Rout[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gp[14];
    pose_epilogue(pose, Fr.R, RB, adj, Rout, v3(0.f, 0.f, 0.f), gp);
    const V3 te = cls == 1 ? a1L - a0L : b1 - b0;
    const float al = cls == 1 ? o.a1 : o.a2;
    const float ex = fmaxf(fmaxf(-al, al - 1.f), 0.f) * k2;
    const int plain = ex * ex * dot(te, te) <= 3600.f;
    for (int i = 0; i < 8; ++i) std::printf("%.9g ", cand.y1[i]);
    std::printf("%.9g ", cand.s1);
    for (int i = 0; i < 8; ++i) std::printf("%.9g ", cand.y2[i]);
    std::printf("%.9g ", cand.s2);
    for (int i = 0; i < 7; ++i) std::printf("%.9g ", gp[i]);
    const V3 dh = cls == 1 ? adj.dB : adj.dA;
    std::printf("%.9g %.9g %.9g %d\n", dh.x, dh.y, dh.z, plain);
  }
  return 0;
}
