// Host build of the kernels' smooth primitive SDFs (prim_sdf: box, capsule,
// cylinder, ellipsoid, from cm_math.cuh) and of their hand-written reverses through
// the SDF normal (normal_bwd, prim_sdf_bwd from cm_adjoint.cuh), for
// tests/test_host_prim_sdf.py.  Reads lines "kind tau y(3) dims(3) phibar nubar(3)"
// (kind 0 box, 1 capsule, 2 cylinder, 3 ellipsoid; dims as the kernels use them)
// and prints per line: phi, the normal nu = g / sqrt(tau + |g|^2) (3), then the
// adjoints of phibar phi + nubar . nu with respect to y (3) and to dims (3).
#include <cstdio>

#include "cm_adjoint.cuh"

using namespace cm;

int main() {
  int kind;
  float tau, v[10];
  while (std::scanf("%d %f", &kind, &tau) == 2) {
    int got = 0;
    for (int i = 0; i < 10; ++i) got += std::scanf("%f", &v[i]);
    if (got != 10) return 2;
    const V3 y = v3(v[0], v[1], v[2]);
    const Body b{kind, v3(v[3], v[4], v[5]), nullptr, 0};
    const float it = 1.f / tau;
    const Sdf f = prim_sdf(b, y, tau, it);
    const V3 nu = normal_of(f.g, tau);
    V3 ybar = v3(0.f, 0.f, 0.f), dbar = v3(0.f, 0.f, 0.f);
    prim_sdf_bwd(b, y, f, tau, it, v[6], normal_bwd(f.g, tau, v3(v[7], v[8], v[9])), ybar, dbar);
    std::printf("%.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g\n", f.phi, nu.x, nu.y, nu.z, ybar.x, ybar.y,
                ybar.z, dbar.x, dbar.y, dbar.z);
  }
  return 0;
}
