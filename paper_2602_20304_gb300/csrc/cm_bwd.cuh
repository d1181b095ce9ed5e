// cm_bwd.cuh -- adjoint kernel of the contact manifold (sm_103a).
//
// Given dL/d out (K x 8 per pair) it returns dL/d poses (14 per pair) and
// dL/d dims (6 per pair).  No candidate of the forward is stored between the
// calls.  With the forward's per-pair record (cm_fwd_kernel given a record
// buffer: the K selected scores, their ids and normalisers, the K rows and the
// soft row / column minima of the E-E distance matrix) a CTA starts from those
// reductions; without it the CTA first recomputes them (candidates, distance
// matrix, nearest-neighbour statistics, the SoftSort top-K list and
// normalisers).  Either way every candidate is then recomputed in the reverse
// sweep:
//   1. SoftSort reverse per candidate (below the K-th score one exponential per
//      candidate, see ss_bwd) -> dL/d(p, d, n, w) and dL/d score, while
//      accumulating dL/d s^_k of the K largest scores; vertex-SDF candidates are
//      backpropagated to the parameters right away;
//   2. each edge pair's reverse (indicators, sign, SDF normals through their
//      Hessian-vector products, witnesses at the fixed QP result) except the
//      nearest-neighbour softmax's coupling across its row and column, kept as
//      t_b = dL/d nn_b * nn_b in the CTA's scratch, summed per row / column, and
//      the QP's own reverse, whose (alpha, con) adjoints are kept per edge pair;
//   3. the K top candidates receive dL/d s^_k through their own score;
//   4. the distance-matrix adjoint dL/d D_kl = (nn1 R_k - t1 + nn2 C_l - t2) / tau
//      flows through |e1* - e2*|, and each edge pair's QP reverse runs once on the
//      sum of its candidates' and its distance's (alpha, con) adjoints;
//   5. CTA reduction of the relative-pose and dims adjoints and the chain to
//      both quaternions and translations.
#pragma once

#include "cm_adjoint.cuh"
#include "cm_pair.cuh"

// The kernel builds are instantiated one per translation unit in cm_bwd_k8.cu,
// cm_bwd_k8b.cu (K <= 8), cm_bwd_k16.cu, cm_bwd_k16b.cu (K <= 16), compiled in
// parallel; cm_bwd.cu dispatches.

namespace cm {

struct BwdShared {
  __align__(16) float G[kMaxK][8];  // upstream of row k in B's frame
  float Gout[kMaxK];  // G_k . out_k
  float invZ[kMaxK];  // 1 / sum_i exp(-|s^_k - s_i| / tau)
  float shat[kMaxK];
  int sid[kMaxK];
  float shatbar[kMaxK];
  // factorised SoftSort reverse below the K-th score r = s^_K (see ss_bwd):
  // c_k = exp((r - s^_k) / tau) / Z_k, Gc = sum_k c_k G_k, cGout = sum_k c_k Gout_k
  __align__(16) float Gc[8];
  float c[kMaxK];
  float cGout, r;
  float Rout[9];      // adjoint of R_B from the output rotation
  float tout[3];
  float adj[18];      // CTA-reduced Adj: R (9), t (3), dA (3), dB (3)
};

// Edge pair (k, l) from the staged endpoint arrays (pre-selected or not).  The
// capsule-template cap signs come with the selected payloads, else from the
// geometry's template rows in global memory.
__device__ __forceinline__ EEGeom ee_geom(const FwdArgs& a, const PairShared& ps, const PairSmem& sm, int k, int l) {
  const int es = sm.es;
  EEGeom g;
  g.a0 = make_float4(sm.eA6[k], sm.eA6[es + k], sm.eA6[2 * es + k], 0.f);
  g.a1 = make_float4(sm.eA6[3 * es + k], sm.eA6[4 * es + k], sm.eA6[5 * es + k], 0.f);
  g.a0L = make_float4(sm.eAl6[k], sm.eAl6[es + k], sm.eAl6[2 * es + k], 0.f);
  g.a1L = make_float4(sm.eAl6[3 * es + k], sm.eAl6[4 * es + k], sm.eAl6[5 * es + k], 0.f);
  g.b0 = make_float4(sm.eB6[l], sm.eB6[es + l], sm.eB6[2 * es + l], 0.f);
  g.b1 = make_float4(sm.eB6[3 * es + l], sm.eB6[4 * es + l], sm.eB6[5 * es + l], 0.f);
  if (ps.kindA == kCapsule) {
    if (ps.kv[2]) {
      const float* v = sel_area(sm).item[2] + 14 * k;
      g.a0L.w = v[12];
      g.a1L.w = v[13];
    } else {
      const uint32_t e = sm.eA[k];
      g.a0L.w = a.verts[ps.voffA + (e & 0xffffu)].w;
      g.a1L.w = a.verts[ps.voffA + (e >> 16)].w;
    }
  }
  if (ps.kindB == kCapsule) {
    if (ps.kv[3]) {
      const float* v = sel_area(sm).item[3] + 8 * l;
      g.b0.w = v[6];
      g.b1.w = v[7];
    } else {
      const uint32_t e = sm.eB[l];
      g.b0.w = a.verts[ps.voffB + (e & 0xffffu)].w;
      g.b1.w = a.verts[ps.voffB + (e >> 16)].w;
    }
  }
  return g;
}

// Per-thread state of the SoftSort reverse: for the candidates below the K-th score,
// E = sum e and Y = sum e y with e = exp((s - r) / tau) (see ss_bwd).  The few at or
// above it add their dL/d s^_k to the CTA's sums directly.
template <int KMAX>
struct SsAcc {
  float E;
  float Y[8];
};

template <int KMAX>
__device__ __forceinline__ void ss_acc_zero(SsAcc<KMAX>& a) {
  a.E = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) a.Y[c] = 0.f;
}

// SoftSort reverse of one candidate (y, s): ybar, sbar and the per-thread partial
// dL/d s^_k.  With G_ki = exp(-|s^_k - s_i| / tau) / Z_k and out_k = sum_i G_ki y_i,
//   ybar_i = sum_k G_ki G_k,  sbar_i = sum_k G_ki (G_k . y_i - G_k . out_k) sgn(s^_k - s_i) / tau,
// and s^_k collects the negated terms.  Below the K-th score r every sign is +1 and
// G_ki = e_i c_k with e_i = exp((s_i - r) / tau), so one exponential serves all K rows:
// ybar_i = e_i Gc, sbar_i = e_i (Gc . y_i - cGout) / tau, and the s^_k terms are summed
// per thread as E and Y and folded in once (ss_finish).  A candidate tied with r whose
// weight w is exactly 0 (an indicator that underflowed, so s = -w d = 0 = r when fewer
// than K scores are positive) takes the same path: ybar is exact (G_ki = c_k), and the
// +1 it gives the tied rows' signs (instead of 0) only reaches w's adjoint and the tied
// rows' s^_k, both of which meet only the underflowed factor's derivative, which is
// exactly 0.  The K top entries and ties with w != 0 (a measure-zero set) take the
// K-row loop, which adds their s^_k terms to bs.shatbar at once.
template <int KMAX>
__device__ __forceinline__ void ss_bwd(BwdShared& bs, int K, float it, float k2, const float (&y)[8], float s,
                                       float (&yb)[8], float& sb, SsAcc<KMAX>& acc) {
  if (s < bs.r || (s == bs.r && y[7] == 0.f)) {
    const float e = ex2((s - bs.r) * k2);
    const float4 g0 = *reinterpret_cast<const float4*>(bs.Gc), g1 = *reinterpret_cast<const float4*>(bs.Gc + 4);
    const float gc[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    float d = -bs.cGout;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      yb[c] = e * gc[c];
      d = fmaf(gc[c], y[c], d);
      acc.Y[c] = fmaf(e, y[c], acc.Y[c]);
    }
    sb = e * d * it;
    acc.E += e;
    return;
  }
  float2 yb2[4] = {dup2(0.f), dup2(0.f), dup2(0.f), dup2(0.f)};
  const float2 yv[4] = {make_float2(y[0], y[1]), make_float2(y[2], y[3]), make_float2(y[4], y[5]),
                        make_float2(y[6], y[7])};
  sb = 0.f;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    if (k < K) {
      const float d = bs.shat[k] - s;
      const float gam = ex2(-fabsf(d) * k2) * bs.invZ[k];
      const float2* G = reinterpret_cast<const float2*>(bs.G[k]);
      float2 a2 = make_float2(-bs.Gout[k], 0.f);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 g = G[c];
        yb2[c] = ffma2(g, dup2(gam), yb2[c]);
        a2 = ffma2(g, yv[c], a2);
      }
      const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      const float term = gam * (a2.x + a2.y) * sg * it;
      sb += term;
      if (term != 0.f) atomicAdd(&bs.shatbar[k], -term);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    yb[2 * c] = yb2[c].x;
    yb[2 * c + 1] = yb2[c].y;
  }
}

__device__ __forceinline__ void adj_reduce(const Adj& a, float* dst) {
  float v[18];
  for (int i = 0; i < 9; ++i) v[i] = a.R[i];
  v[9] = a.t.x; v[10] = a.t.y; v[11] = a.t.z;
  v[12] = a.dA.x; v[13] = a.dA.y; v[14] = a.dA.z;
  v[15] = a.dB.x; v[16] = a.dB.y; v[17] = a.dB.z;
#pragma unroll
  for (int i = 0; i < 18; ++i) {
    float s = warp_sum(v[i]);
    if ((threadIdx.x & 31) == 0) atomicAdd(&dst[i], s);
  }
}


// Everything the reverse phases of one pair read.
struct BwdPair {
  const FwdArgs* a;
  const PairShared* ps;
  PairSmem sm;
  BwdShared* bs;
  Frame F;
  PairBodies bb;
  float *Dm, *T1, *T2, *QA1, *QA2, *QCN, *rowR, *colC;
  float* QB;          // per edge pair: the QP result's adjoints (alpha1, alpha2, con) at QB[c * qbs + i]
  int64_t qbs;
  int nvs, neB, nee, K;
  float* sadj;  // pre-selection adjoint slots (null when nothing is selected)
};

// Export slots of the pre-selected items (see kSelAdjFloats): A's vertices,
// B's vertices, A's edges, B's edges, then the vertex-depth adjoints of A and B.
__device__ __forceinline__ float* vexp_of(const BwdPair& P, int c) {
  if (!P.sadj) return nullptr;
  if (c < P.ps->nvA) return P.ps->kv[0] ? P.sadj + 3 * c : nullptr;
  return P.ps->kv[1] ? P.sadj + 3 * kMaxSel + 3 * (c - P.ps->nvA) : nullptr;
}
__device__ __forceinline__ float* eAexp_of(const BwdPair& P, int k) {
  return P.sadj && P.ps->kv[2] ? P.sadj + 6 * kMaxSel + 6 * k : nullptr;
}
__device__ __forceinline__ float* eBexp_of(const BwdPair& P, int l) {
  return P.sadj && P.ps->kv[3] ? P.sadj + 12 * kMaxSel + 6 * l : nullptr;
}

// Folds the below-threshold sums into dL/d s^_k (-c_k (G_k . Y - Gout_k E) / tau) and
// adds the warp's totals to the CTA's.
template <int KMAX>
__device__ __forceinline__ void ss_finish(SsAcc<KMAX>& acc, int K, float it, BwdShared& bs) {
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    if (k < K) {
      float d = -bs.Gout[k] * acc.E;
#pragma unroll
      for (int c = 0; c < 8; ++c) d = fmaf(bs.G[k][c], acc.Y[c], d);
      const float v = warp_sum(-bs.c[k] * d * it);
      if ((threadIdx.x & 31) == 0) atomicAdd(&bs.shatbar[k], v);
    }
  }
}

// Vertex-SDF reverse of this thread's candidates.
template <int KMAX, int kCls>
__device__ __forceinline__ void vs_reverse_phase(const BwdPair P) {
  const PairShared& ps = *P.ps;
  Adj adj;
  adj_zero(adj);
  SsAcc<KMAX> acc;
  ss_acc_zero(acc);
  float y[8];
  for (int c = threadIdx.x; c < P.nvs; c += blockDim.x) {
    const float s = vs_candidate(ps, P.sm, P.bb, c, y);
    float yb[8], sb;
    ss_bwd<KMAX>(*P.bs, P.K, P.F.inv_tau, P.F.k2, y, s, yb, sb, acc);
    if (c < ps.nvA)
      vs_bwd<true, kCls>(P.F, P.bb.A, P.bb.B, P.sm.vAl[c], ld3(P.sm.vA[c]), yb, sb, adj, vexp_of(P, c));
    else
      vs_bwd<false, kCls>(P.F, P.bb.A, P.bb.B, P.sm.vB[c - ps.nvA], ld3(P.sm.vB[c - ps.nvA]), yb, sb, adj,
                          vexp_of(P, c));
  }
  ss_finish<KMAX>(acc, P.K, P.F.inv_tau, *P.bs);
  adj_reduce(adj, P.bs->adj);
}

// The k-th selected score passes dL/d s^_k to its own candidate.
template <int kCls>
__device__ __forceinline__ void fixup_phase(const BwdPair P, const int k) {
  const PairShared& ps = *P.ps;
  const int id = P.bs->sid[k];
  const float sx = P.bs->shatbar[k];
  const float zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  Adj adj;
  adj_zero(adj);
  if (id >= 0 && id < P.nvs) {
    if (id < ps.nvA) vs_bwd<true, kCls>(P.F, P.bb.A, P.bb.B, P.sm.vAl[id], ld3(P.sm.vA[id]), zero, sx, adj, vexp_of(P, id));
    else
      vs_bwd<false, kCls>(P.F, P.bb.A, P.bb.B, P.sm.vB[id - ps.nvA], ld3(P.sm.vB[id - ps.nvA]), zero, sx, adj,
                    vexp_of(P, id));
  } else if (id >= P.nvs) {
    const int e = id - P.nvs, i = e >> 1, b = e & 1, kk = i / P.neB, ll = i - kk * P.neB;
    float t1, t2;
    const QPOut qs{P.QA1[i], P.QA2[i], P.QCN[i]};
    const QPBar qb = ee_bwd<kCls>(P.F, P.bb.A, P.bb.B, P.a->p, ee_geom(*P.a, ps, P.sm, kk, ll), P.sm.rowL[kk],
                                        P.sm.colL[ll], &qs,
           [&](const EECand&, float (&yb1)[8], float& sb1, float (&yb2)[8], float& sb2) {
             for (int c = 0; c < 8; ++c) {
               yb1[c] = 0.f;
               yb2[c] = 0.f;
             }
             sb1 = b == 0 ? sx : 0.f;
             sb2 = b == 1 ? sx : 0.f;
           },
           t1, t2, adj, eAexp_of(P, kk), eBexp_of(P, ll));
    atomicAdd(&P.T1[i], t1);
    atomicAdd(&P.T2[i], t2);
    atomicAdd(&P.rowR[kk], t1);
    atomicAdd(&P.colC[ll], t2);
    atomicAdd(&P.QB[i], qb.a1);
    atomicAdd(&P.QB[P.qbs + i], qb.a2);
    atomicAdd(&P.QB[2 * P.qbs + i], qb.con);
  }
  float* dst = P.bs->adj;
  for (int i = 0; i < 9; ++i) atomicAdd(&dst[i], adj.R[i]);
  atomicAdd(&dst[9], adj.t.x); atomicAdd(&dst[10], adj.t.y); atomicAdd(&dst[11], adj.t.z);
  atomicAdd(&dst[12], adj.dA.x); atomicAdd(&dst[13], adj.dA.y); atomicAdd(&dst[14], adj.dA.z);
  atomicAdd(&dst[15], adj.dB.x); atomicAdd(&dst[16], adj.dB.y); atomicAdd(&dst[17], adj.dB.z);
}

// Last pass over the edge pairs: the distance-matrix adjoint through the
// nearest-neighbour softmaxes, then each edge pair's QP reverse once, on the sum of
// its candidates' and its distance's (alpha, con) adjoints.
template <int kCls>
__device__ __forceinline__ void qp_phase(const BwdPair P) {
  Adj adj;
  adj_zero(adj);
  const float k2 = P.F.k2, it = P.F.inv_tau;
  for (int i = threadIdx.x; i < P.nee; i += blockDim.x) {
    const int k = i / P.neB, l = i - k * P.neB;
    const float D = P.Dm[i];
    const float nn1 = ex2((P.sm.rowL[k] - D) * k2), nn2 = ex2((P.sm.colL[l] - D) * k2);
    const float Db = (nn1 * P.rowR[k] - P.T1[i] + nn2 * P.colC[l] - P.T2[i]) * it;
    const QPOut qs{P.QA1[i], P.QA2[i], P.QCN[i]};
    const QPBar qb{P.QB[i], P.QB[P.qbs + i], P.QB[2 * P.qbs + i]};
    ee_qp_bwd<kCls>(P.F, P.bb.A, P.bb.B, P.a->p, ee_geom(*P.a, *P.ps, P.sm, k, l), Db, qs, qb, adj, eAexp_of(P, k),
                    eBexp_of(P, l));
  }
  adj_reduce(adj, P.bs->adj);
}

// Reverse of the four soft selections (one warp each): the items' local-frame
// payload adjoints xbar_k give every item's score adjoint through
// Gamma_ki = exp(-|s^_k - s_i| / tau) / Z_k (and s^_k through the k-th top
// item), and scores pass to the vertex depths (-m for a vertex, -(m_0 + m_1)/2
// for an edge).  Needs the pair's original vertices / edges staged again.
static __device__ __forceinline__ void sel_reverse_phase(const BwdPair P) {
  const PairShared& ps = *P.ps;
  const PairSmem& sm = P.sm;
  const SelArea A = sel_area(sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float* mbar[2] = {P.sadj + kSelAdjFloats, P.sadj + kSelAdjFloats + sm.vs};
  const float k2 = P.F.k2, it = P.F.inv_tau;
  const int es = sm.es;
  // score adjoint of item i of selection `kind` -> depth adjoints
  auto to_depths = [&](int kind, int i, float sbar) {
    if (kind < 2) {
      atomicAdd(&mbar[kind][i], -sbar);
    } else {
      const uint32_t e = kind == 2 ? sm.eA[i] : sm.eB[i];
      atomicAdd(&mbar[kind - 2][e & 0xffffu], -0.5f * sbar);
      atomicAdd(&mbar[kind - 2][e >> 16], -0.5f * sbar);
    }
  };
  for (int kind = warp; kind < 4; kind += nwarps) {
    const int K = ps.kv[kind];
    if (!K) continue;
    const int n = kind == 0 ? ps.nvA0 : kind == 1 ? ps.nvB0 : kind == 2 ? ps.neA0 : ps.neB0;
    const int P3 = kind < 2 ? 3 : 6;                       // local payload width
    const int off = kind == 0 ? 3 : kind == 1 ? 0 : kind == 2 ? 6 : 0;  // local part in the payload
    const float* xb = P.sadj + (kind == 0 ? 0 : kind == 1 ? 3 * kMaxSel : kind == 2 ? 6 * kMaxSel : 12 * kMaxSel);
    const float* item = A.item[kind];
    const float* info = A.info[kind];
    const int W = sel_width(kind);
    for (int k = 0; k < K; ++k) {
      const float sh = info[k], iz = 1.f / info[kMaxSel + k];
      const float* xk = xb + P3 * k;
      float xs = 0.f;  // xbar_k . x_sel_k
      for (int c = 0; c < P3; ++c) xs = fmaf(xk[c], item[W * k + off + c], xs);
      float shb = 0.f;
      for (int i = lane; i < n; i += 32) {
        const float si = sel_score(sm, A, kind, i);
        float xi[6];
        if (kind == 0) {
          const float4 v = sm.vAl[i];
          xi[0] = v.x; xi[1] = v.y; xi[2] = v.z;
        } else if (kind == 1) {
          const float4 v = sm.vB[i];
          xi[0] = v.x; xi[1] = v.y; xi[2] = v.z;
        } else {
          const float* src = kind == 2 ? sm.eAl6 : sm.eB6;
          for (int c = 0; c < 6; ++c) xi[c] = src[c * es + i];
        }
        float ax = -xs;
        for (int c = 0; c < P3; ++c) ax = fmaf(xk[c], xi[c], ax);
        const float d = sh - si;
        const float gam = ex2(-fabsf(d) * k2) * iz;
        const float t = gam * ax * (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * it;
        if (t != 0.f) to_depths(kind, i, t);
        shb -= t;
      }
      shb = warp_sum(shb);
      if (lane == 0 && shb != 0.f) to_depths(kind, __float_as_int(info[2 * kMaxSel + k]), shb);
    }
  }
}

// Depth adjoints: m_A[i] = phi_B(v_i) for A's original vertices and
// m_B[j] = phi_A(v_j) for B's, back to both poses and dims.
static __device__ __forceinline__ void depth_adjoint_phase(const BwdPair P) {
  const PairShared& ps = *P.ps;
  const PairSmem& sm = P.sm;
  const float* mbarA = P.sadj + kSelAdjFloats;
  const float* mbarB = mbarA + sm.vs;
  const float tau = P.F.tau, it = P.F.inv_tau;
  Adj adj;
  adj_zero(adj);
  for (int i = threadIdx.x; i < ps.nvA0 + ps.nvB0; i += blockDim.x) {
    if (i < ps.nvA0) {
      const float mb = mbarA[i];
      if (mb == 0.f) continue;
      const V3 y = ld3(sm.vA[i]);
      const float4 vL = sm.vAl[i];
      const Sdf f = body_sdf(P.bb.B, y, tau, it);
      V3 yb = v3(0.f, 0.f, 0.f);
      body_sdf_bwd(P.bb.B, y, f, tau, it, mb, v3(0.f, 0.f, 0.f), yb, adj.dB);
      const V3 vl = v3(vL.x, vL.y, vL.z);
      const V3 vb = push_point_bwd(P.F, vl, yb, adj);
      map_vertex_bwd(ps.kindA, vl, vL.w, P.bb.A.dims, vb, adj.dA);
    } else {
      const int j = i - ps.nvA0;
      const float mb = mbarB[j];
      if (mb == 0.f) continue;
      const float4 vv = sm.vB[j];
      const V3 y = v3(vv.x, vv.y, vv.z);
      const V3 x = mulT(P.F.R, y - P.F.t);
      const Sdf f = body_sdf(P.bb.A, x, tau, it);
      V3 xb = v3(0.f, 0.f, 0.f);
      body_sdf_bwd(P.bb.A, x, f, tau, it, mb, v3(0.f, 0.f, 0.f), xb, adj.dA);
      const V3 pb = pull_point_bwd(P.F, y, xb, adj);
      map_vertex_bwd(ps.kindB, y, vv.w, P.bb.B.dims, pb, adj.dB);
    }
  }
  adj_reduce(adj, P.bs->adj);
}

// The reverse sweep's pass over the edge pairs (step 2 of the header) for pair class
// kCls (0: any kinds; 1: A a hull and B a primitive, see sdf2h_of): the QP (solved here
// when the forward's record is read), both candidates, their SoftSort reverse and the
// rest of the element's reverse, keeping t1, t2 and the QP adjoints per edge pair.
template <int KMAX, int kCls>
__device__ __forceinline__ void ee_reverse_pass(const BwdPair& P, BwdShared& bs, const float* rec, int64_t ss) {
  const FwdArgs& a = *P.a;
  const PairShared& ps = *P.ps;
  const PairSmem& sm = P.sm;
  const int K = P.K, neB = P.neB, nee = P.nee;
  const float it = P.F.inv_tau, k2 = P.F.k2;
  float *Dm = P.Dm, *T1 = P.T1, *T2 = P.T2, *QA1 = P.QA1, *QA2 = P.QA2, *QCN = P.QCN, *QB = P.QB;
  float *rowR = P.rowR, *colC = P.colC;
  Adj adj;
  adj_zero(adj);
  SsAcc<KMAX> acc;
  ss_acc_zero(acc);
  for (int i = threadIdx.x; i < nee; i += blockDim.x) {
    const int k = i / neB, l = i - k * neB;
    const EEGeom gg = ee_geom(a, ps, sm, k, l);
    QPOut qs;
    if (rec) {  // the QP result and the distance matrix for the last pass
      qs = qp_solve(qp_setup(xyz(gg.a0), xyz(gg.a1), xyz(gg.b0), xyz(gg.b1), a.p.w_reg), a.p.w_reg, a.p);
      QA1[i] = qs.a1;
      QA2[i] = qs.a2;
      QCN[i] = qs.con;
    } else {
      qs = QPOut{QA1[i], QA2[i], QCN[i]};
    }
    float t1, t2;
    const QPBar qb = ee_bwd<kCls>(P.F, P.bb.A, P.bb.B, a.p, gg, sm.rowL[k], sm.colL[l], &qs,
           [&](const EECand& cc, float (&yb1)[8], float& sb1, float (&yb2)[8], float& sb2) {
             // both candidates through one copy of the SoftSort reverse
#pragma unroll 1
             for (int j = 0; j < 2; ++j) {
               float yc[8], yb[8], sb;
#pragma unroll
               for (int c = 0; c < 8; ++c) yc[c] = j ? cc.y2[c] : cc.y1[c];
               ss_bwd<KMAX>(bs, K, it, k2, yc, j ? cc.s2 : cc.s1, yb, sb, acc);
#pragma unroll
               for (int c = 0; c < 8; ++c) {
                 if (j) yb2[c] = yb[c];
                 else yb1[c] = yb[c];
               }
               if (j) sb2 = sb;
               else sb1 = sb;
             }
           },
           t1, t2, adj, eAexp_of(P, k), eBexp_of(P, l), rec ? Dm + i : nullptr);
    T1[i] = t1;
    T2[i] = t2;
    QB[i] = qb.a1;
    QB[ss + i] = qb.a2;
    QB[2 * ss + i] = qb.con;
    atomicAdd(&rowR[k], t1);
    atomicAdd(&colC[l], t2);
  }
  ss_finish<KMAX>(acc, K, it, bs);
  adj_reduce(adj, bs.adj);
}

template <int kMinBlocks, int KMAX>
__global__ void __launch_bounds__(256, kMinBlocks) cm_bwd_kernel(const FwdArgs a, const float* grad_out,
                                                                 float* grad_poses, float* grad_dims) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairShared ps;
  __shared__ BwdShared bs;
  const PairSmem sm = carve(smem_raw, a.sm);
  float* rowR = sm.rowL + a.sm.max_e;  // second half of the statistics buffers
  float* colC = sm.colL + a.sm.max_e;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int K = a.p.K;
  const int64_t ss = a.scratch_stride;
  float* Dm = a.scratch + (int64_t)blockIdx.x * ss * kBwdScratchArrays;
  float* T1 = Dm + ss;
  float* T2 = T1 + ss;
  float* QA1 = T2 + ss;  // alpha1, alpha2, con of every edge pair
  float* QA2 = QA1 + ss;
  float* QCN = QA2 + ss;
  float* QB = QCN + ss;  // their adjoints (3 arrays)
  int iter = 0;
  for (;;) {
    const int pi = next_pair(a, iter);
    if (pi < 0) break;
    __syncthreads();
    if (threadIdx.x == 0) pair_setup(a, pi, ps);
    __syncthreads();
    if (ps.bad) {
      if (threadIdx.x == 0) atomicCAS(a.err, 0, pi + 1);
      for (int i = threadIdx.x; i < 14; i += blockDim.x) grad_poses[(size_t)pi * 14 + i] = __int_as_float(0x7fc00000);
      if (grad_dims)
        for (int i = threadIdx.x; i < 6; i += blockDim.x) grad_dims[(size_t)pi * 6 + i] = __int_as_float(0x7fc00000);
      continue;
    }
    pair_stage(a, pi, ps, sm);
    __syncthreads();
    const PairBodies bb = pair_bodies(ps, sm);
    float* sadj = nullptr;
    if (ps.preselect) {
      preselect_pair(a, ps, sm, bb);
      sadj = sm.sadj;
      for (int i = threadIdx.x; i < kSelAdjFloats + 2 * sm.vs; i += blockDim.x) sadj[i] = 0.f;
    }
    const float k2 = ps.k2, it = ps.inv_tau;
    Frame F;
    F.R = ps.Rrel;
    F.t = ps.trel;
    F.tau = ps.tau;
    F.inv_tau = it;
    F.k2 = k2;
    const bool one_sided = (a.p.flags & 2) != 0;
    const bool no_ee = one_sided || (a.p.flags & 1) != 0;
    const int nvs = one_sided ? ps.nvA : ps.nvA + ps.nvB;
    const int neA = ps.neA, neB = ps.neB, nee = no_ee ? 0 : neA * neB;
    // the forward's record of this pair (cm_fwd_kernel with a record buffer), if any
    const float* rec = a.saved ? a.saved + (size_t)pi * a.saved_stride : nullptr;

    // ================= the forward's top-K list and nearest-neighbour statistics
    float y[8], Z = 1.f, ls = -3.0e38f;
    int lid = -1;
    if (rec) {
      if (nee) {
        for (int k = threadIdx.x; k < neA; k += blockDim.x) {
          sm.rowL[k] = rec[kRecHead * K + k];
          rowR[k] = 0.f;
        }
        for (int l = threadIdx.x; l < neB; l += blockDim.x) {
          sm.colL[l] = rec[kRecHead * K + a.sm.max_e + l];
          colC[l] = 0.f;
        }
      }
      if (warp == 0 && lane < K) {
        ls = rec[lane];
        lid = __float_as_int(rec[K + lane]);
        Z = rec[2 * K + lane];
        for (int c = 0; c < 8; ++c) y[c] = rec[3 * K + 8 * lane + c];
      }
    } else {  // recompute the pair's forward
      WarpTopK st;
      wtk_init(st, sm.warp + warp * kWarpStateFloats);
      float y2[8];
      for (int base = warp * 32; base < nvs; base += nwarps * 32) {
        const int c = base + lane;
        const bool valid = c < nvs;
        float s = 0.f;
        if (valid) s = vs_candidate(ps, sm, bb, c, y);
        wtk_push(st, valid, s, y, K, k2, c);
      }
      if (nee) {
        for (int i = threadIdx.x; i < nee; i += blockDim.x) {
          const int k = i / neB, l = i - k * neB;
          const Witness w = ee_witness(edge_pair(sm, k, l), a.p);
          Dm[i] = w.dbar;
          QA1[i] = w.qp.a1;
          QA2[i] = w.qp.a2;
          QCN[i] = w.qp.con;
        }
        __syncthreads();
        for (int k = warp; k < neA; k += nwarps) {
          float m = 3.0e38f;
          for (int l = lane; l < neB; l += 32) m = fminf(m, Dm[k * neB + l]);
          m = warp_min(m);
          float S = 0.f;
          for (int l = lane; l < neB; l += 32) S += ex2((m - Dm[k * neB + l]) * k2);
          S = warp_sum(S);
          if (lane == 0) {
            sm.rowL[k] = m - ps.tau * kLn2 * lg2(S);
            rowR[k] = 0.f;
          }
        }
        for (int l = threadIdx.x; l < neB; l += blockDim.x) {
          float m = 3.0e38f;
          for (int k = 0; k < neA; ++k) m = fminf(m, Dm[k * neB + l]);
          float S = 0.f;
          for (int k = 0; k < neA; ++k) S += ex2((m - Dm[k * neB + l]) * k2);
          sm.colL[l] = m - ps.tau * kLn2 * lg2(S);
          colC[l] = 0.f;
        }
        __syncthreads();
        for (int base = warp * 32; base < nee; base += nwarps * 32) {
          const int i = base + lane;
          const bool valid = i < nee;
          float s1 = 0.f, s2 = 0.f;
          if (valid) {
            const int k = i / neB, l = i - k * neB;
            const EdgePair ep = edge_pair(sm, k, l);
            const Witness w = ee_witness_from(ep, QPOut{QA1[i], QA2[i], QCN[i]});
            ee_candidates(ps, sm, bb, ep, w, sm.rowL[k], sm.colL[l], y, y2, s1, s2);
          }
          wtk_push(st, valid, s1, y, K, k2, nvs + 2 * i);
          wtk_push(st, valid, s2, y2, K, k2, nvs + 2 * i + 1);
        }
      }
      // merge the warps' states pairwise (log2(nwarps) levels)
      for (int h = 1; h < nwarps; h <<= 1) {
        if ((warp & (2 * h - 1)) == h) wtk_store(st, K);
        __syncthreads();
        if ((warp & (2 * h - 1)) == 0 && warp + h < nwarps) wtk_merge(st, sm.warp + (warp + h) * kWarpStateFloats, K, k2);
      }
      if (warp == 0) {
        wtk_finish(st, K, k2, y, &Z);
        ls = st.ls;
        lid = st.lid;
      }
    }
    if (warp == 0) {
      // upstream of row k in B's frame and the output-rotation adjoints
      float Rl[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      V3 tl = v3(0.f, 0.f, 0.f);
      if (lane < K) {
        const float* g = grad_out + ((size_t)pi * K + lane) * 8;
        V3 gp = v3(g[0], g[1], g[2]), gn = v3(g[4], g[5], g[6]);
        V3 gpb = mulT(ps.RB, gp), gnb = mulT(ps.RB, gn);
        float G[8] = {gpb.x, gpb.y, gpb.z, g[3], gnb.x, gnb.y, gnb.z, g[7]};
        float go = 0.f;
        for (int c = 0; c < 8; ++c) {
          bs.G[lane][c] = G[c];
          go = fmaf(G[c], y[c], go);
        }
        bs.Gout[lane] = go;
        bs.invZ[lane] = 1.0f / Z;
        bs.shat[lane] = ls;
        bs.sid[lane] = lid;
        bs.shatbar[lane] = 0.f;
        add_outer(Rl, gp, v3(y[0], y[1], y[2]));
        add_outer(Rl, gn, v3(y[4], y[5], y[6]));
        tl = gp;
      }
      // constants of the factorised SoftSort reverse below the K-th score r
      const float r = __shfl_sync(kFull, ls, K - 1);
      const float ck = lane < K ? ex2((r - ls) * k2) * (1.0f / Z) : 0.f;
      float gcs = 0.f;
      for (int c = 0; c < 8; ++c) {
        const float v = warp_sum(lane < K ? ck * bs.G[lane][c] : 0.f);
        if (lane == c) gcs = v;
      }
      if (lane < 8) bs.Gc[lane] = gcs;
      const float cgo = warp_sum(lane < K ? ck * bs.Gout[lane] : 0.f);
      if (lane < K) bs.c[lane] = ck;
      if (lane == 0) {
        bs.cGout = cgo;
        bs.r = r;
      }
      for (int i = 0; i < 9; ++i) Rl[i] = warp_sum(Rl[i]);
      tl = v3(warp_sum(tl.x), warp_sum(tl.y), warp_sum(tl.z));
      if (lane == 0) {
        for (int i = 0; i < 9; ++i) bs.Rout[i] = Rl[i];
        bs.tout[0] = tl.x; bs.tout[1] = tl.y; bs.tout[2] = tl.z;
      }
    }
    for (int i = threadIdx.x; i < 18; i += blockDim.x) bs.adj[i] = 0.f;
    __syncthreads();

    // ================= reverse sweep
    BwdPair P;
    P.a = &a;
    P.ps = &ps;
    P.sm = sm;
    P.bs = &bs;
    P.F = F;
    P.bb = bb;
    P.Dm = Dm; P.T1 = T1; P.T2 = T2; P.QA1 = QA1; P.QA2 = QA2; P.QCN = QCN; P.rowR = rowR; P.colC = colC;
    P.QB = QB;
    P.qbs = ss;
    P.nvs = nvs; P.neB = neB; P.nee = nee; P.K = K;
    P.sadj = sadj;
    // a hull against a primitive (either way round) runs code specialised for it
    const int cls = (ps.kindA == kHull && ps.kindB <= kEllipsoid) ? 1
                    : (ps.kindA <= kEllipsoid && ps.kindB == kHull) ? 2 : 0;
    if (cls == 1) {
      vs_reverse_phase<KMAX, 1>(P);
      ee_reverse_pass<KMAX, 1>(P, bs, rec, ss);
    } else if (cls == 2) {
      vs_reverse_phase<KMAX, 2>(P);
      ee_reverse_pass<KMAX, 2>(P, bs, rec, ss);
    } else {
      vs_reverse_phase<KMAX, 0>(P);
      ee_reverse_pass<KMAX, 0>(P, bs, rec, ss);
    }
    __syncthreads();
    {  // selected candidate k on lane k / nwarps of warp k % nwarps: each warp runs its
       // own candidates' reverse, so vertex and edge candidates do not serialise in one warp
      const int k = lane * nwarps + warp;
      if (k < K) {
        if (cls == 1) fixup_phase<1>(P, k);
        else if (cls == 2) fixup_phase<2>(P, k);
        else fixup_phase<0>(P, k);
      }
    }
    __syncthreads();
    if (cls == 1) qp_phase<1>(P);
    else if (cls == 2) qp_phase<2>(P);
    else qp_phase<0>(P);
    __syncthreads();
    if (sadj) {  // pre-selection: stage the original geometry again, then its reverse
      if (threadIdx.x == 0) {
        ps.nvA = ps.nvA0; ps.nvB = ps.nvB0; ps.neA = ps.neA0; ps.neB = ps.neB0;
      }
      __syncthreads();
      pair_stage(a, pi, ps, sm);
      __syncthreads();
      sel_reverse_phase(P);
      __syncthreads();
      depth_adjoint_phase(P);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      Adj r;
      for (int i = 0; i < 9; ++i) r.R[i] = bs.adj[i];
      r.t = v3(bs.adj[9], bs.adj[10], bs.adj[11]);
      r.dA = v3(bs.adj[12], bs.adj[13], bs.adj[14]);
      r.dB = v3(bs.adj[15], bs.adj[16], bs.adj[17]);
      float gp[14];
      pose_epilogue(a.poses + 14 * (size_t)pi, ps.RA, ps.RB, r, bs.Rout, v3(bs.tout[0], bs.tout[1], bs.tout[2]), gp);
      for (int i = 0; i < 14; ++i) grad_poses[(size_t)pi * 14 + i] = gp[i];
      if (grad_dims) {
        float* gd = grad_dims + (size_t)pi * 6;
        gd[0] = r.dA.x; gd[1] = r.dA.y; gd[2] = r.dA.z;
        gd[3] = r.dB.x; gd[4] = r.dB.y; gd[5] = r.dB.z;
      }
    }
  }
}

// Builds of the adjoint kernel: one CTA per SM with up to 255 registers, or two
// CTAs per SM within 128 registers (spilling to L1; the launch shape's CTAs per
// SM picks: 1 -> the first); each for K <= 8 and K <= 16 (the SoftSort reverse
// unrolls to it).
// Dynamic shared memory the two builds are configured for: the two-CTA build
// takes layouts up to kBwdSmem2, larger ones run the one-CTA build.
constexpr int kBwdSmem1 = 180 * 1024, kBwdSmem2 = 110 * 1024;

template <int MB, int KM>
cudaError_t launch_bwd_t(const FwdArgs& a, const float* g, float* gp, float* gd, int grid, int block,
                                cudaStream_t s) {
  cudaError_t e = ensure_smem_attr(reinterpret_cast<const void*>(cm_bwd_kernel<MB, KM>),
                                   MB == 1 ? kBwdSmem1 : kBwdSmem2);
  if (e != cudaSuccess) return e;
  cm_bwd_kernel<MB, KM><<<grid, block, a.sm.total, s>>>(a, g, gp, gd);
  return cudaGetLastError();
}

}  // namespace cm
