// Host build of the kernels' superquadric-union SDF (sdf_sq_union, cm_math.cuh) and
// its hand-written reverse through the normal (normal_bwd, sdf_sq_union_bwd,
// cm_adjoint.cuh) for tests/test_host_sq_union.py.  Input: "tau L", then L rows of the
// union as the C ABI takes them (qw qx qy qz tx ty tz eps1 a b c eps2: orientation,
// centre, semi-axes and exponents), then lines "y(3) phibar nubar(3)".  The rows are
// packed here as geometry registration packs them for the kernels: the rows of R^T
// with -R^T t, then (1/a, 1/b, 1/c, 2/eps1) and (2/eps2, eps2/eps1, eps1/2, 0).
// Output per line: phi, the normal nu = g / sqrt(tau + |g|^2) (3) and the adjoint of
// phibar phi + nubar . nu with respect to y (3).
#include <cmath>
#include <cstdio>
#include <vector>

#include "cm_adjoint.cuh"

using namespace cm;

int main() {
  float tau;
  int L;
  if (std::scanf("%f %d", &tau, &L) != 2 || L <= 0) return 2;
  std::vector<float4> P;
  for (int l = 0; l < L; ++l) {
    double r[12];
    for (int i = 0; i < 12; ++i)
      if (std::scanf("%lf", &r[i]) != 1) return 2;
    const double n = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    const double w = r[0] / n, x = r[1] / n, y = r[2] / n, z = r[3] / n;
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    for (int i = 0; i < 3; ++i) {
      const double c = -(R[0][i] * r[4] + R[1][i] * r[5] + R[2][i] * r[6]);
      P.push_back(make_float4((float)R[0][i], (float)R[1][i], (float)R[2][i], (float)c));
    }
    P.push_back(make_float4((float)(1.0 / r[8]), (float)(1.0 / r[9]), (float)(1.0 / r[10]), (float)(2.0 / r[7])));
    P.push_back(make_float4((float)(2.0 / r[11]), (float)(r[11] / r[7]), (float)(0.5 * r[7]), 0.f));
  }
  float v[7];
  for (;;) {
    int got = 0;
    for (int i = 0; i < 7; ++i) got += std::scanf("%f", &v[i]);
    if (got != 7) break;
    const V3 y = v3(v[0], v[1], v[2]);
    const Sdf f = sdf_sq_union(y, P.data(), L, tau, 1.f / tau);
    const V3 nu = normal_of(f.g, tau);
    V3 ybar = v3(0.f, 0.f, 0.f);
    sdf_sq_union_bwd(y, P.data(), L, f, 1.f / tau, v[3], normal_bwd(f.g, tau, v3(v[4], v[5], v[6])), ybar);
    std::printf("%.9g %.9g %.9g %.9g %.9g %.9g %.9g\n", f.phi, nu.x, nu.y, nu.z, ybar.x, ybar.y, ybar.z);
  }
  return 0;
}
