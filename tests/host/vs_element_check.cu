// Host build of the adjoint's vertex-SDF element (vs_bwd: a vertex of one body
// against the other body's smooth SDF, Sec. IV-C, reversed by hand; pose_epilogue:
// the chain to the quaternion and translation) for tests/test_host_vs_element.py, on
// the kernels' hull-vs-primitive pair class: A a convex polyhedron, B a box at the
// origin, unrotated.  Input: "tau F", F plane rows (n_x n_y n_z c, A's frame), then per
// line: side (0: a vertex of A against B, 1: a vertex of B against A) qA(4) tA(3) v(3)
// (A's local vertex, or B's box template row) hB(3) yb(8) sb (upstream adjoints of the
// row (p, d, n, w) and of the score s = -w d).  Output per line: the gradient of
// yb . row + sb s with respect to qA(4), tA(3) and hB(3).
#include <cstdio>
#include <vector>

#include "cm_adjoint.cuh"

using namespace cm;

int main() {
  float tau;
  int F;
  if (std::scanf("%f %d", &tau, &F) != 2 || F <= 0) return 2;
  const float k2 = kLog2e / tau;
  std::vector<float4> P(F);
  for (int f = 0; f < F; ++f) {
    float x, y, z, c;
    if (std::scanf("%f %f %f %f", &x, &y, &z, &c) != 4) return 2;
    P[f] = make_float4(k2 * x, k2 * y, k2 * z, k2 * c);  // staged as base-2 exponents
  }
  int side;
  float v[22];
  while (std::scanf("%d", &side) == 1) {
    int got = 0;
    for (int i = 0; i < 22; ++i) got += std::scanf("%f", &v[i]);
    if (got != 22) return 2;
    const float pose[14] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], 1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    Frame Fr;
    Fr.R = quat_rot(v[0], v[1], v[2], v[3]);
    Fr.t = v3(v[4], v[5], v[6]);
    Fr.tau = tau;
    Fr.inv_tau = 1.f / tau;
    Fr.k2 = k2;
    const V3 hB = v3(v[10], v[11], v[12]);
    const Body A{kHull, v3(1.f, 1.f, 1.f), P.data(), F};
    const Body B{kBox, hB, nullptr, 0};
    float yb[8];
    for (int i = 0; i < 8; ++i) yb[i] = v[13 + i];
    Adj adj;
    adj_zero(adj);
    if (side == 0) {
      const V3 vl = v3(v[7], v[8], v[9]);
      vs_bwd<true, 1>(Fr, A, B, make_float4(vl.x, vl.y, vl.z, 0.f), mul(Fr.R, vl) + Fr.t, yb, v[21], adj);
    } else {
      const V3 vb = v3(v[7] * hB.x, v[8] * hB.y, v[9] * hB.z);
      vs_bwd<false, 1>(Fr, A, B, make_float4(v[7], v[8], v[9], 0.f), vb, yb, v[21], adj);
    }
    const M3 RB = quat_rot(1.f, 0.f, 0.f, 0.f);
    const float Rout[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gp[14];
    pose_epilogue(pose, Fr.R, RB, adj, Rout, v3(0.f, 0.f, 0.f), gp);
    for (int i = 0; i < 7; ++i) std::printf("%.9g ", gp[i]);
    std::printf("%.9g %.9g %.9g\n", adj.dB.x, adj.dB.y, adj.dB.z);
  }
  return 0;
}
