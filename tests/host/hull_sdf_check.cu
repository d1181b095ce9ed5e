// Host build of the kernels' polyhedron SDF routines (cm_math.cuh compiled for the
// CPU: the MUFU wrappers fall back to exp2f / log2f / division) for
// tests/test_host_hull_sdf.py.  Reads from stdin: tau, the plane count F, F rows
// (n_x n_y n_z c) of unit normals and offsets, then lines "y1x y1y y1z y2x y2y y2z";
// for each point pair prints both routines' outputs on one line:
//   shifted (sdf_planes2_h): phi1 g1(3) phi2 g2(3) H(6), then plain (sdf_planes2_h_ee): the same.
#include <cstdio>
#include <vector>

#include "cm_math.cuh"

using namespace cm;

static void put(const Sdf& a, const Sdf& b, const float (&H)[6]) {
  std::printf(" %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g", a.phi, a.g.x, a.g.y, a.g.z, b.phi, b.g.x, b.g.y, b.g.z);
  for (int i = 0; i < 6; ++i) std::printf(" %.9g", H[i]);
}

int main() {
  float tau;
  int F;
  if (std::scanf("%f %d", &tau, &F) != 2 || F <= 0) return 2;
  const float k = kLog2e / tau;  // planes pre-scaled to base-2 exponents, as the kernels stage them
  std::vector<float4> P(F);
  for (int f = 0; f < F; ++f) {
    float nx, ny, nz, c;
    if (std::scanf("%f %f %f %f", &nx, &ny, &nz, &c) != 4) return 2;
    P[f] = make_float4(k * nx, k * ny, k * nz, k * c);
  }
  float a[6];
  while (std::scanf("%f %f %f %f %f %f", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5]) == 6) {
    const V3 y1 = v3(a[0], a[1], a[2]), y2 = v3(a[3], a[4], a[5]);
    Sdf s1, s2, p1, p2;
    float Hs[6], Hp[6];
    sdf_planes2_h(y1, y2, P.data(), F, tau, s1, s2, Hs);
    sdf_planes2_h_ee(y1, y2, P.data(), F, tau, p1, p2, Hp);
    put(s1, s2, Hs);
    put(p1, p2, Hp);
    std::printf("\n");
  }
  return 0;
}
