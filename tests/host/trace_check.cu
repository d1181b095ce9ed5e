// Host build of the kernels' sphere tracing of a witness (trace_to_surface,
// cm_math.cuh) and its hand-written reverse (trace_bwd, cm_adjoint.cuh) for
// tests/test_host_trace.py.  Input: "kind tau iters F" (kind 0 box, 1 capsule,
// 2 cylinder, 3 ellipsoid, 4 convex polyhedron; F plane rows n_x n_y n_z c follow for
// a polyhedron, F = 0 otherwise), then lines "x0(3) dims(3) xbar(3)".  Output per line:
// the traced point (3), then the adjoints of xbar . x_traced with respect to x0 (3) and
// to dims (3).
#include <cstdio>
#include <vector>

#include "cm_adjoint.cuh"

using namespace cm;

int main() {
  int kind, iters, F;
  float tau;
  if (std::scanf("%d %f %d %d", &kind, &tau, &iters, &F) != 4 || iters < 1 || iters > 8) return 2;
  const float k2 = kLog2e / tau;
  std::vector<float4> P(F > 0 ? F : 1);
  for (int f = 0; f < F; ++f) {
    float x, y, z, c;
    if (std::scanf("%f %f %f %f", &x, &y, &z, &c) != 4) return 2;
    P[f] = make_float4(k2 * x, k2 * y, k2 * z, k2 * c);  // staged as base-2 exponents
  }
  float v[9];
  for (;;) {
    int got = 0;
    for (int i = 0; i < 9; ++i) got += std::scanf("%f", &v[i]);
    if (got != 9) break;
    const Body b{kind, v3(v[3], v[4], v[5]), P.data(), F};
    const V3 x0 = v3(v[0], v[1], v[2]);
    const V3 x = trace_to_surface(b, x0, iters, tau, 1.f / tau);
    V3 dbar = v3(0.f, 0.f, 0.f);
    const V3 xb = trace_bwd(b, x0, iters, tau, 1.f / tau, v3(v[6], v[7], v[8]), dbar);
    std::printf("%.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g\n", x.x, x.y, x.z, xb.x, xb.y, xb.z, dbar.x, dbar.y,
                dbar.z);
  }
  return 0;
}
