// cm_fwd_warp.cu -- forward contact-manifold kernel for small pairs: one warp per
// pair (sm_103a).
//
// A pair of small bodies (a box has 8 vertices, 12 edges and 144 edge pairs against
// another box) leaves most of a CTA idle and pays a CTA barrier per phase in
// cm_fwd_kernel.  Here each warp owns one pair at a time, with its own slice of
// shared memory: the pair's staged geometry, the E-E distance matrix and QP results
// of every edge pair (4 floats each) and its SoftSort state.  The phases are those
// of cm_fwd_kernel (Sec. IV-C vertex candidates; Sec. IV-D2 QP pass; the soft row
// and column minima behind the nearest-neighbour indicators of Sec. IV-D3; the
// edge candidates; the SoftSort reduction of Sec. III), separated by warp
// synchronisation only; with a single SoftSort state per pair nothing is merged.
// Records for the adjoint and the candidate dump are written as cm_fwd_kernel
// writes them.  Pre-selection is not supported here (its selection is CTA-wide).
#include "cm_pair.cuh"

namespace cm {

__device__ __forceinline__ void warp_dump_row(const FwdArgs& a, const PairShared& ps, int64_t row,
                                              const float (&y)[8]) {
  const V3 p = mul(ps.RB, v3(y[0], y[1], y[2])) + ps.tB;
  const V3 n = mul(ps.RB, v3(y[4], y[5], y[6]));
  float* o = a.dump + row * 8;
  o[0] = p.x; o[1] = p.y; o[2] = p.z; o[3] = y[3];
  o[4] = n.x; o[5] = n.y; o[6] = n.z; o[7] = y[7];
}

constexpr int kWarpKernelMaxWarps = 8;

// warp_bytes: one warp's slice of dynamic shared memory, the single-warp SmemLayout
// (a.sm) followed by 4 max_e^2 floats (distance, alpha1, alpha2, con per edge pair).
__global__ void __launch_bounds__(256) cm_fwd_warp_kernel(const FwdArgs a, int warp_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairShared ps_all[kWarpKernelMaxWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned char* base = smem_raw + (size_t)warp * warp_bytes;
  const PairSmem sm = carve(base, a.sm);
  const int ee_cap = a.sm.max_e * a.sm.max_e;
  float* D = reinterpret_cast<float*>(base + a.sm.total);
  float* QA1 = D + ee_cap;
  float* QA2 = QA1 + ee_cap;
  float* QCN = QA2 + ee_cap;
  PairShared& ps = ps_all[warp];
  const int K = a.p.K;
  const bool one_sided = (a.p.flags & 2) != 0;
  const bool no_ee = one_sided || (a.p.flags & 1) != 0;
  const int gw = blockIdx.x * nwarps + warp, nw = gridDim.x * nwarps;
  for (int it = 0;; ++it) {
    int n;
    if (a.work_counter) {
      n = 0;
      if (lane == 0) n = atomicAdd(a.work_counter, 1);
      n = __shfl_sync(kFull, n, 0);
    } else {
      n = gw + it * nw;
    }
    if (n >= a.n_pairs) break;
    const int pi = a.order ? a.order[n] : n;
    __syncwarp();
    if (lane == 0) pair_setup(a, pi, ps);
    __syncwarp();
    if (ps.bad) {
      if (lane == 0) atomicCAS(a.err, 0, pi + 1);
      for (int i = lane; i < K * 8; i += 32) a.out[(size_t)pi * K * 8 + i] = __int_as_float(0x7fc00000);
      continue;
    }
    pair_stage_by(a, pi, ps, sm, lane, 32);
    __syncwarp();
    const PairBodies bb = pair_bodies(ps, sm);
    const float k2 = ps.k2;
    const int nvs = one_sided ? ps.nvA : ps.nvA + ps.nvB;
    const int neA = ps.neA, neB = ps.neB, nee = no_ee ? 0 : neA * neB;
    int64_t doff = -1;
    if (a.dump) {
      const int64_t o0 = a.dump_off[pi], o1 = a.dump_off[pi + 1];
      if (o0 >= 0 && o1 - o0 == nvs + 2 * (int64_t)nee && o1 <= a.dump_rows) doff = o0;
      else if (lane == 0) atomicCAS(a.err, 0, -(pi + 1));
    }

    WarpTopK st;
    wtk_init(st, sm.warp);
    float y[8], y2[8];
    for (int b0 = 0; b0 < nvs; b0 += 32) {
      const int c = b0 + lane;
      const bool valid = c < nvs;
      float s = 0.f;
      if (valid) {
        s = vs_candidate(ps, sm, bb, c, y);
        if (doff >= 0) warp_dump_row(a, ps, doff + c, y);
      }
      wtk_push(st, valid, s, y, K, k2, c);
    }
    if (nee) {
      // QP of every edge pair: distance and result kept in the warp's slice
      for (int i = lane; i < nee; i += 32) {
        const int k = i / neB, l = i - k * neB;
        const Witness w = ee_witness(edge_pair(sm, k, l), a.p);
        D[i] = w.dbar;
        QA1[i] = w.qp.a1;
        QA2[i] = w.qp.a2;
        QCN[i] = w.qp.con;
      }
      __syncwarp();
      // soft row and column minima, a lane per row / column
      for (int k = lane; k < neA; k += 32) {
        float m = 3.0e38f;
        for (int l = 0; l < neB; ++l) m = fminf(m, D[k * neB + l]);
        float S = 0.f;
        for (int l = 0; l < neB; ++l) S += ex2((m - D[k * neB + l]) * k2);
        sm.rowL[k] = m - ps.tau * kLn2 * lg2(S);
      }
      for (int l = lane; l < neB; l += 32) {
        float m = 3.0e38f;
        for (int k = 0; k < neA; ++k) m = fminf(m, D[k * neB + l]);
        float S = 0.f;
        for (int k = 0; k < neA; ++k) S += ex2((m - D[k * neB + l]) * k2);
        sm.colL[l] = m - ps.tau * kLn2 * lg2(S);
      }
      __syncwarp();
      if (a.saved && pi >= a.saved_first) {
        float* rec = a.saved + (size_t)(pi - a.saved_first) * a.saved_stride + kRecHead * K;
        for (int k = lane; k < neA; k += 32) rec[k] = sm.rowL[k];
        for (int l = lane; l < neB; l += 32) rec[a.sm.max_e + l] = sm.colL[l];
      }
      for (int b0 = 0; b0 < nee; b0 += 32) {
        const int i = b0 + lane;
        const bool valid = i < nee;
        float s1 = 0.f, s2 = 0.f;
        if (valid) {
          const int k = i / neB, l = i - k * neB;
          const EdgePair ep = edge_pair(sm, k, l);
          const Witness w = ee_witness_from(ep, QPOut{QA1[i], QA2[i], QCN[i]});
          ee_candidates(ps, sm, bb, ep, w, sm.rowL[k], sm.colL[l], y, y2, s1, s2);
          if (doff >= 0) {
            warp_dump_row(a, ps, doff + nvs + 2 * (int64_t)i, y);
            warp_dump_row(a, ps, doff + nvs + 2 * (int64_t)i + 1, y2);
          }
        }
        wtk_push(st, valid, s1, y, K, k2, nvs + 2 * i);
        wtk_push(st, valid, s2, y2, K, k2, nvs + 2 * i + 1);
      }
    }
    float Z = 1.f;
    wtk_finish(st, K, k2, y, &Z);
    if (a.saved && pi >= a.saved_first && lane < K) {
      float* rec = a.saved + (size_t)(pi - a.saved_first) * a.saved_stride;
      rec[lane] = st.ls;
      rec[K + lane] = __int_as_float(st.lid);
      rec[2 * K + lane] = Z;
      for (int c = 0; c < 8; ++c) rec[3 * K + 8 * lane + c] = y[c];
    }
    if (lane < K) {
      const V3 p = mul(ps.RB, v3(y[0], y[1], y[2])) + ps.tB;
      const V3 nn = mul(ps.RB, v3(y[4], y[5], y[6]));
      float* o = a.out + ((size_t)pi * K + lane) * 8;
      o[0] = p.x; o[1] = p.y; o[2] = p.z; o[3] = y[3];
      o[4] = nn.x; o[5] = nn.y; o[6] = nn.z; o[7] = y[7];
    }
  }
}

constexpr int kFwdWarpSmemMax = 200 * 1024;

int fwd_warp_bytes(const SmemLayout& L) {
  return ((L.total + 15) & ~15) + 16 * L.max_e * L.max_e;
}

cudaError_t launch_fwd_warp(const FwdArgs& a, int grid, int block, cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cm_fwd_warp_kernel), kFwdWarpSmemMax);
  if (e != cudaSuccess) return e;
  const int wb = fwd_warp_bytes(a.sm);
  cm_fwd_warp_kernel<<<grid, block, (size_t)wb * (block / 32), s>>>(a, wb);
  return cudaGetLastError();
}

int fwd_warp_max_blocks_per_sm(int block, int smem_bytes) {
  int n = 0;
  if (ensure_smem_attr(reinterpret_cast<const void*>(cm_fwd_warp_kernel), kFwdWarpSmemMax) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cm_fwd_warp_kernel, block, smem_bytes) != cudaSuccess) return 0;
  return n;
}

bool fwd_warp_fits(const SmemLayout& L, int block) {
  return (size_t)fwd_warp_bytes(L) * (block / 32) <= (size_t)kFwdWarpSmemMax && block / 32 <= kWarpKernelMaxWarps;
}

}  // namespace cm
