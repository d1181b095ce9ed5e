// cm_witness.cu -- batched witness-point routines on their own (the paper's
// witness-point throughput setting): independent edge-edge or vertex-triangle
// queries, one thread each, 48-byte rows read as three float4 and results
// written as float4.
#include "contact_manifold.h"
#include "cm_internal.h"
#include "cm_context.h"

namespace cm {
namespace {

// kHard: the non-smoothed active set (the paper's Ours-NS, Sec. V)
template <bool kHard>
__global__ void __launch_bounds__(256) ee_witness_kernel(int n, const float4* __restrict__ q, Params p,
                                                         float4* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 r0 = q[3 * i], r1 = q[3 * i + 1], r2 = q[3 * i + 2];
    const V3 a0 = v3(r0.x, r0.y, r0.z), a1 = v3(r0.w, r1.x, r1.y), b0 = v3(r1.z, r1.w, r2.x),
             b1 = v3(r2.y, r2.z, r2.w);
    const QPPre pre = qp_setup(a0, a1, b0, b1, p.w_reg);
    const QPOut o = kHard ? qp_solve_hard(pre, p.w_reg) : qp_solve(pre, p.w_reg, p);
    const V3 e1 = fma3(o.a1, a1 - a0, a0), e2 = fma3(o.a2, b1 - b0, b0);
    const V3 d = e1 - e2;
    out[2 * i] = make_float4(e1.x, e1.y, e1.z, e2.x);
    out[2 * i + 1] = make_float4(e2.y, e2.z, o.con, sqrt_(dot(d, d)));
  }
}

template <bool kHard>
__global__ void __launch_bounds__(256) vf_witness_kernel(int n, const float4* __restrict__ q, Params p,
                                                         float4* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 r0 = q[3 * i], r1 = q[3 * i + 1], r2 = q[3 * i + 2];
    float inside;
    const V3 v = v3(r0.x, r0.y, r0.z), t0 = v3(r0.w, r1.x, r1.y), t1 = v3(r1.z, r1.w, r2.x),
             t2 = v3(r2.y, r2.z, r2.w);
    const V3 w = kHard ? vf_witness_hard(v, t0, t1, t2, inside) : vf_witness(v, t0, t1, t2, p, inside);
    out[i] = make_float4(w.x, w.y, w.z, inside);
  }
}

int grid_for(int n) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (n + 255) / 256;
  return blocks < sms * 8 ? (blocks > 0 ? blocks : 1) : sms * 8;
}

cm_status check_batch(int32_t n, const void* q, const cm_params* params, const void* out) {
  cm_status st = rt::check_params(params);
  if (st != CM_OK) return st;
  if (n < 0) return rt::fail(CM_ERR_INVALID_ARG, "n < 0");
  if (n > 0 && (!q || !out)) return rt::fail(CM_ERR_INVALID_ARG, "queries and out are required");
  if (((uintptr_t)q | (uintptr_t)out) & 15) return rt::fail(CM_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  return CM_OK;
}

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" cm_status cm_ee_witness_batch(int32_t n, const float* queries, const cm_params* params, float* out,
                                         void* stream) {
  cm_status st = check_batch(n, queries, params, out);
  if (st != CM_OK || n == 0) return st;
  const Params p{params->tau, params->w_reg, params->eps_clip, params->eps_min, params->eps_comp, params->K,
                 params->flags, 0, 0};
  const float4* q4 = reinterpret_cast<const float4*>(queries);
  float4* o4 = reinterpret_cast<float4*>(out);
  if (params->flags & CM_FLAG_HARD) ee_witness_kernel<true><<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, q4, p, o4);
  else ee_witness_kernel<false><<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, q4, p, o4);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CM_OK : rt::cuda_fail(e, "E-E witness launch");
}

extern "C" cm_status cm_vf_witness_batch(int32_t n, const float* queries, const cm_params* params, float* out,
                                         void* stream) {
  cm_status st = check_batch(n, queries, params, out);
  if (st != CM_OK || n == 0) return st;
  const Params p{params->tau, params->w_reg, params->eps_clip, params->eps_min, params->eps_comp, params->K,
                 params->flags, 0, 0};
  const float4* q4 = reinterpret_cast<const float4*>(queries);
  float4* o4 = reinterpret_cast<float4*>(out);
  if (params->flags & CM_FLAG_HARD) vf_witness_kernel<true><<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, q4, p, o4);
  else vf_witness_kernel<false><<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, q4, p, o4);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CM_OK : rt::cuda_fail(e, "V-F witness launch");
}
