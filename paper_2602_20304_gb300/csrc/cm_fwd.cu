// cm_fwd.cu -- forward contact-manifold kernel (sm_103a).
//
// One CTA per body pair at a time (a persistent grid walks a work queue of
// pairs).  Per pair:
//   1. stage both meshes and A's planes/B's planes in shared memory, A moved
//      into B's frame;
//   2. vertex-SDF candidates (Sec. IV-C), warp-strided from the last warp down,
//      streamed into the warp's SoftSort top-K state;
//   3. E-E pass 1: witness QP of every edge pair -> unsigned distance dbar_kl and
//      the QP result, kept in the CTA's scratch slice (global memory, L2-resident),
//      and each column's minimum (shared-memory atomicMin);
//   4. soft row and column minima L = m - tau log sum exp(-(dbar - m)/tau) of
//      the distance matrix (nn indicators of Sec. IV-D3, Eq. nn_check): one sweep,
//      a warp per row, also adds the column sums;
//   5. E-E pass 2: witnesses from the kept QP results, four SDF evaluations,
//      sign, pen, nn, cl and activity -> two candidates per edge pair, streamed
//      into the warp state;
//   6. merge the warps' states pairwise and write the K rows, rotated back to world.
// With a record buffer the pair's selected list, its normalisers and rows and the
// soft row / column minima are also written for the adjoint (cm_bwd_kernel), which
// then needs no recompute of the forward's reductions.
#include "cm_pair.cuh"

namespace cm {

// One candidate row (p, d, n, w) of the dump, rotated back to world coordinates.
__device__ __forceinline__ void dump_row(const FwdArgs& a, const PairShared& ps, int64_t row, const float (&y)[8]) {
  const V3 p = mul(ps.RB, v3(y[0], y[1], y[2])) + ps.tB;
  const V3 n = mul(ps.RB, v3(y[4], y[5], y[6]));
  float* o = a.dump + row * 8;
  o[0] = p.x; o[1] = p.y; o[2] = p.z; o[3] = y[3];
  o[4] = n.x; o[5] = n.y; o[6] = n.z; o[7] = y[7];
}

__global__ void __launch_bounds__(512) cm_fwd_kernel(const FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairShared ps;
  const PairSmem sm = carve(smem_raw, a.sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int K = a.p.K;
  const int64_t ss = a.scratch_stride;
  float* D = a.scratch + (int64_t)blockIdx.x * ss * (a.store_alpha ? 4 : 1);
  float* A1 = D + ss;   // alpha1, alpha2, con of pass 1 (store_alpha only)
  float* A2 = A1 + ss;
  float* CN = A2 + ss;
  int it = 0;
  for (;;) {
    const int pi = next_pair(a, it);
    if (pi < 0) break;
    __syncthreads();
    if (threadIdx.x == 0) pair_setup(a, pi, ps);
    __syncthreads();
    if (ps.bad) {
      if (threadIdx.x == 0) atomicCAS(a.err, 0, pi + 1);
      for (int i = threadIdx.x; i < K * 8; i += blockDim.x) a.out[(size_t)pi * K * 8 + i] = __int_as_float(0x7fc00000);
      continue;
    }
    pair_stage(a, pi, ps, sm);
    // row and column statistics of the E-E distance matrix: running minima (as the
    // bits of non-negative floats) and the column soft-minimum sums
    float* colS = sm.colL + a.sm.max_e;
    for (int l = threadIdx.x; l < ps.neB; l += blockDim.x) {
      sm.colL[l] = 3.0e38f;
      colS[l] = 0.f;
    }
    for (int k = threadIdx.x; k < ps.neA; k += blockDim.x) sm.rowL[k] = 3.0e38f;
    __syncthreads();
    const PairBodies bb = pair_bodies(ps, sm);
    if (ps.preselect) preselect_pair(a, ps, sm, bb);
    const float k2 = ps.k2;

    WarpTopK st;
    wtk_init(st, sm.warp + warp * kWarpStateFloats);
    float y[8], y2[8];

    // ---- vertex-SDF candidates, from the last warp down: the thread-strided E-E
    // pass 1 gives its extra elements to the first warps
    const bool one_sided = (a.p.flags & 2) != 0;
    const bool no_ee = one_sided || (a.p.flags & 1) != 0;
    const int nvs = one_sided ? ps.nvA : ps.nvA + ps.nvB;
    // candidate dump: this pair's rows start at dump_off[pi], one per candidate id; a
    // range that does not match the pair's candidate count or the buffer is refused
    int64_t doff = -1;
    if (a.dump) {
      const int64_t o0 = a.dump_off[pi], o1 = a.dump_off[pi + 1];
      const int64_t total = nvs + (no_ee ? 0 : 2 * (int64_t)ps.neA * ps.neB);
      if (o0 >= 0 && o1 - o0 == total && o1 <= a.dump_rows) doff = o0;
      else if (threadIdx.x == 0) atomicCAS(a.err, 0, -(pi + 1));
    }
    for (int base = (nwarps - 1 - warp) * 32; base < nvs; base += nwarps * 32) {
      const int c = base + lane;
      const bool valid = c < nvs;
      float s = 0.f;
      if (valid) {
        s = vs_candidate(ps, sm, bb, c, y);
        if (doff >= 0) dump_row(a, ps, doff + c, y);
      }
      wtk_push(st, valid, s, y, K, k2, c);
    }

    if (!no_ee) {
      const int neA = ps.neA, neB = ps.neB, nee = neA * neB;
      // ---- E-E pass 1: unsigned distances
      for (int i = threadIdx.x; i < nee; i += blockDim.x) {
        const int k = i / neB, l = i - k * neB;
        Witness w = ee_witness(edge_pair(sm, k, l), a.p);
        D[i] = w.dbar;
        atomicMin(reinterpret_cast<int*>(sm.colL) + l, __float_as_int(w.dbar));
        atomicMin(reinterpret_cast<int*>(sm.rowL) + k, __float_as_int(w.dbar));
        if (a.store_alpha) {
          A1[i] = w.qp.a1;
          A2[i] = w.qp.a2;
          CN[i] = w.qp.con;
        }
      }
      __syncthreads();
      // ---- soft row minima (warp per row, coalesced over the row) and, in the same
      // sweep, the column sums, both against the minima found in pass 1
      for (int k = warp; k < neA; k += nwarps) {
        const float m = sm.rowL[k];
        float S = 0.f;
        for (int l = lane; l < neB; l += 32) {
          const float d = D[k * neB + l];
          S += ex2((m - d) * k2);
          atomicAdd(colS + l, ex2((sm.colL[l] - d) * k2));
        }
        S = warp_sum(S);
        if (lane == 0) sm.rowL[k] = m - ps.tau * kLn2 * lg2(S);
      }
      __syncthreads();
      for (int l = threadIdx.x; l < neB; l += blockDim.x) sm.colL[l] -= ps.tau * kLn2 * lg2(colS[l]);
      __syncthreads();
      if (a.saved && pi >= a.saved_first) {  // the soft minima go to the pair's record for the adjoint
        float* rec = a.saved + (size_t)(pi - a.saved_first) * a.saved_stride + kRecHead * K;
        for (int k = threadIdx.x; k < neA; k += blockDim.x) rec[k] = sm.rowL[k];
        for (int l = threadIdx.x; l < neB; l += blockDim.x) rec[a.sm.max_e + l] = sm.colL[l];
      }
      // ---- E-E pass 2: candidates
      for (int base = warp * 32; base < nee; base += nwarps * 32) {
        const int i = base + lane;
        const bool valid = i < nee;
        float s1 = 0.f, s2 = 0.f;
        if (valid) {
          const int k = i / neB, l = i - k * neB;
          const EdgePair ep = edge_pair(sm, k, l);
          Witness w;
          if (a.store_alpha) {
            QPOut q;
            q.a1 = A1[i];
            q.a2 = A2[i];
            q.con = CN[i];
            w = ee_witness_from(ep, q);
          } else {
            w = ee_witness(ep, a.p);
          }
          ee_candidates(ps, sm, bb, ep, w, sm.rowL[k], sm.colL[l], y, y2, s1, s2);
          if (doff >= 0) {
            dump_row(a, ps, doff + nvs + 2 * (int64_t)i, y);
            dump_row(a, ps, doff + nvs + 2 * (int64_t)i + 1, y2);
          }
        }
        wtk_push(st, valid, s1, y, K, k2, nvs + 2 * i);
        wtk_push(st, valid, s2, y2, K, k2, nvs + 2 * i + 1);
      }
    }

    // ---- merge the warps' states pairwise (log2(nwarps) levels) and write the K rows
    for (int h = 1; h < nwarps; h <<= 1) {
      if ((warp & (2 * h - 1)) == h) wtk_store(st, K);
      __syncthreads();
      if ((warp & (2 * h - 1)) == 0 && warp + h < nwarps) wtk_merge(st, sm.warp + (warp + h) * kWarpStateFloats, K, k2);
    }
    if (warp == 0) {
      float Z = 1.f;
      wtk_finish(st, K, k2, y, &Z);
      if (a.saved && pi >= a.saved_first && lane < K) {  // the selected list and its rows (B's frame)
        float* rec = a.saved + (size_t)(pi - a.saved_first) * a.saved_stride;
        rec[lane] = st.ls;
        rec[K + lane] = __int_as_float(st.lid);
        rec[2 * K + lane] = Z;
        for (int c = 0; c < 8; ++c) rec[3 * K + 8 * lane + c] = y[c];
      }
      if (lane < K) {
        V3 p = mul(ps.RB, v3(y[0], y[1], y[2])) + ps.tB;
        V3 n = mul(ps.RB, v3(y[4], y[5], y[6]));
        float* o = a.out + ((size_t)pi * K + lane) * 8;
        o[0] = p.x; o[1] = p.y; o[2] = p.z; o[3] = y[3];
        o[4] = n.x; o[5] = n.y; o[6] = n.z; o[7] = y[7];
      }
    }
  }
}

constexpr int kFwdSmemMax = 200 * 1024;

cudaError_t launch_fwd(const FwdArgs& a, int grid, int block, cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cm_fwd_kernel), kFwdSmemMax);
  if (e != cudaSuccess) return e;
  cm_fwd_kernel<<<grid, block, a.sm.total, s>>>(a);
  return cudaGetLastError();
}

int fwd_max_blocks_per_sm(int block, int smem_bytes) {
  int n = 0;
  if (ensure_smem_attr(reinterpret_cast<const void*>(cm_fwd_kernel), kFwdSmemMax) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cm_fwd_kernel, block, smem_bytes) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

}  // namespace cm
