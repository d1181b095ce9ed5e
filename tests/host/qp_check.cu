// Host build of the kernels' edge-edge box QP (qp_setup + qp_solve from
// cm_math.cuh) and its hand-written reverse (qp_bwd from cm_adjoint.cuh), for
// tests/test_host_qp.py.  Reads lines "a0 a1 b0 b1 abar1 abar2 conbar" (12 + 3
// numbers: the two edges' endpoints and the adjoints of alpha1, alpha2, con) and
// prints per line: alpha1 alpha2 con, then the endpoint adjoints a0 a1 b0 b1
// (12 numbers) of abar1 alpha1 + abar2 alpha2 + conbar con.  Parameters are the
// method's defaults: w_reg = 0.01, eps_clip = eps_min = eps_comp = 0.1.
#include <cstdio>

#include "cm_adjoint.cuh"

using namespace cm;

int main() {
  Params p{};
  p.tau = 1e-2f;
  p.w_reg = 0.01f;
  p.eps_clip = p.eps_min = p.eps_comp = 0.1f;
  p.K = 8;
  float v[15];
  for (;;) {
    int got = 0;
    for (int i = 0; i < 15; ++i) got += std::scanf("%f", &v[i]);
    if (got != 15) break;
    const V3 a0 = v3(v[0], v[1], v[2]), a1 = v3(v[3], v[4], v[5]);
    const V3 b0 = v3(v[6], v[7], v[8]), b1 = v3(v[9], v[10], v[11]);
    const QPPre q = qp_setup(a0, a1, b0, b1, p.w_reg);
    const QPOut o = qp_solve(q, p.w_reg, p);
    V3 a0b = v3(0.f, 0.f, 0.f), a1b = a0b, b0b = a0b, b1b = a0b;
    qp_bwd(q, p.w_reg, p, v[12], v[13], v[14], a0b, a1b, b0b, b1b);
    std::printf("%.9g %.9g %.9g", o.a1, o.a2, o.con);
    for (const V3& g : {a0b, a1b, b0b, b1b}) std::printf(" %.9g %.9g %.9g", g.x, g.y, g.z);
    std::printf("\n");
  }
  return 0;
}
