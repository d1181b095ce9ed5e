// cm_pair.cuh -- per-pair staging and per-candidate arithmetic shared by the
// forward and adjoint kernels.
//
// A CTA owns one body pair at a time.  Everything is evaluated in the local
// frame of body B: B's vertices and planes are used as registered, A's
// vertices are moved by the relative pose (R_rel = R_B^T R_A,
// t_rel = R_B^T (t_A - t_B)), and A's SDF at a B-frame point y is evaluated at
// R_rel^T (y - t_rel) in A's frame.  Outputs are rotated back to world at the end.
#pragma once

#include "cm_internal.h"
#include "cm_softsort.cuh"

namespace cm {

static_assert(kSsFloats <= kWarpStateFloats && kMaxK <= 16, "per-warp SoftSort area");

struct PairShared {
  M3 RA, RB, Rrel;
  V3 tA, tB, trel;
  V3 dA, dB;
  int kindA, kindB;
  int nvA, nvB, neA, neB, npA, npB;
  float tau, inv_tau, k2;
  int bad;  // invalid geometry id
  int preselect;  // soft pre-selection active for this pair
  int trace;      // sphere-tracing steps of E-E witnesses
  int nvA0, nvB0, neA0, neB0;  // counts before pre-selection
  int kv[4];                   // selected counts (0: that selection is off)
  int voffA, voffB;            // template rows of A and B in the vertex store
};

struct PairSmem {
  float4* vA;      // A's vertices in B's frame
  float4* vAl;     // A's vertices in A's own frame
  float4* vB;      // B's vertices (B frame = local)
  float4* pA;      // A's planes (A frame)
  float4* pB;      // B's planes
  uint32_t* eA;
  uint32_t* eB;
  float* eA6;      // A's edge endpoints in B's frame, SoA: [c * max_e + k], c = a0x, a0y, a0z, a1x, a1y, a1z
  float* eAl6;     // A's edge endpoints in A's frame, same layout
  float* eB6;      // B's edge endpoints, same layout
  float* sel;      // pre-selection: vertex depths of A and B, then the staged soft selections
  float* sadj;     // adjoint kernel only: pre-selection adjoint slots (kSelAdjFloats + 2 vs)
  int es;          // SoA stride (largest edge count)
  int vs;          // vertex stride (largest vertex count)
  float* rowL;     // soft row minima of the E-E distance matrix (nn-Gamma_1)
  float* colL;     // soft column minima (nn-Gamma_2)
  float* warp;     // per-warp SoftSort states
};

__device__ __forceinline__ PairSmem carve(unsigned char* base, const SmemLayout& L) {
  PairSmem s;
  s.vA = reinterpret_cast<float4*>(base + L.vA);
  s.vAl = reinterpret_cast<float4*>(base + L.vAl);
  s.vB = reinterpret_cast<float4*>(base + L.vB);
  s.pA = reinterpret_cast<float4*>(base + L.pA);
  s.pB = reinterpret_cast<float4*>(base + L.pB);
  s.eA = reinterpret_cast<uint32_t*>(base + L.eA);
  s.eB = reinterpret_cast<uint32_t*>(base + L.eB);
  s.rowL = reinterpret_cast<float*>(base + L.rowL);
  s.colL = reinterpret_cast<float*>(base + L.colL);
  s.warp = reinterpret_cast<float*>(base + L.warp);
  s.eA6 = reinterpret_cast<float*>(base + L.eA6);
  s.eAl6 = reinterpret_cast<float*>(base + L.eAl6);
  s.eB6 = reinterpret_cast<float*>(base + L.eB6);
  s.sel = reinterpret_cast<float*>(base + L.sel);
  s.sadj = reinterpret_cast<float*>(base + L.sadj);
  s.es = L.max_e;
  s.vs = L.max_v;
  return s;
}

// Thread 0: header, pose and frame set-up of pair `pi`.  Returns via `ps`.
__device__ inline void pair_setup(const FwdArgs& a, int pi, PairShared& ps) {
  const int ga = a.pair_geoms[2 * pi], gb = a.pair_geoms[2 * pi + 1];
  ps.bad = (ga < 0 || ga >= a.n_geoms || gb < 0 || gb >= a.n_geoms) ? 1 : 0;
  if (ps.bad) return;
  const GeomHeader& A = a.hdr[ga];
  const GeomHeader& B = a.hdr[gb];
  if (A.n_verts <= 0 || B.n_verts <= 0) {  // destroyed geometry (cm_destroy_geometry)
    ps.bad = 1;
    return;
  }
  const float* P = a.poses + 14 * (size_t)pi;
  ps.RA = quat_rot(P[0], P[1], P[2], P[3]);
  ps.tA = v3(P[4], P[5], P[6]);
  ps.RB = quat_rot(P[7], P[8], P[9], P[10]);
  ps.tB = v3(P[11], P[12], P[13]);
  ps.Rrel = mulTM(ps.RB, ps.RA);
  ps.trel = mulT(ps.RB, ps.tA - ps.tB);
  if (a.dims) {
    const float* D = a.dims + 6 * (size_t)pi;
    ps.dA = v3(D[0], D[1], D[2]);
    ps.dB = v3(D[3], D[4], D[5]);
  } else {
    ps.dA = v3(A.dims[0], A.dims[1], A.dims[2]);
    ps.dB = v3(B.dims[0], B.dims[1], B.dims[2]);
  }
  ps.kindA = A.kind;
  ps.kindB = B.kind;
  ps.nvA = A.n_verts; ps.nvB = B.n_verts;
  ps.neA = A.n_edges; ps.neB = B.n_edges;
  ps.npA = A.n_planes; ps.npB = B.n_planes;
  ps.preselect = (a.p.top_verts > 0 || a.p.top_edges > 0) ? 1 : 0;
  ps.trace = a.p.trace_iters;
  ps.nvA0 = ps.nvA; ps.nvB0 = ps.nvB; ps.neA0 = ps.neA; ps.neB0 = ps.neB;
  ps.kv[0] = ps.kv[1] = ps.kv[2] = ps.kv[3] = 0;
  ps.voffA = A.v_off;
  ps.voffB = B.v_off;
  ps.tau = a.tau ? a.tau[pi] : a.p.tau;
  ps.inv_tau = 1.0f / ps.tau;
  ps.k2 = ps.inv_tau * kLog2e;
}

// Cooperative: copy pair `pi`'s geometry into shared memory (A's vertices moved
// into B's frame), thread t0 of a group of ts threads (the CTA, or one warp).
// Caller syncs the group before and after.
__device__ inline void pair_stage_by(const FwdArgs& a, int pi, const PairShared& ps, const PairSmem& sm, int t0,
                                     int ts) {
  const int ga = a.pair_geoms[2 * pi], gb = a.pair_geoms[2 * pi + 1];
  const GeomHeader& A = a.hdr[ga];
  const GeomHeader& B = a.hdr[gb];
  for (int i = t0; i < ps.nvA; i += ts) {
    float4 u = a.verts[A.v_off + i];
    V3 v = map_vertex(ps.kindA, u.x, u.y, u.z, u.w, ps.dA);
    V3 y = mul(ps.Rrel, v) + ps.trel;
    sm.vA[i] = make_float4(y.x, y.y, y.z, 0.f);
    sm.vAl[i] = make_float4(v.x, v.y, v.z, u.w);  // w: template cap sign (capsules)
  }
  for (int i = t0; i < ps.nvB; i += ts) {
    float4 u = a.verts[B.v_off + i];
    V3 v = map_vertex(ps.kindB, u.x, u.y, u.z, u.w, ps.dB);
    sm.vB[i] = make_float4(v.x, v.y, v.z, u.w);
  }
  for (int i = t0; i < ps.neA; i += ts) {
    const uint32_t e = a.edges[A.e_off + i];
    sm.eA[i] = e;
    const float4 u0 = a.verts[A.v_off + (e & 0xffffu)], u1 = a.verts[A.v_off + (e >> 16)];
    const V3 l0 = map_vertex(ps.kindA, u0.x, u0.y, u0.z, u0.w, ps.dA);
    const V3 l1 = map_vertex(ps.kindA, u1.x, u1.y, u1.z, u1.w, ps.dA);
    const V3 w0 = mul(ps.Rrel, l0) + ps.trel, w1 = mul(ps.Rrel, l1) + ps.trel;
    const int es = sm.es;
    sm.eA6[i] = w0.x; sm.eA6[es + i] = w0.y; sm.eA6[2 * es + i] = w0.z;
    sm.eA6[3 * es + i] = w1.x; sm.eA6[4 * es + i] = w1.y; sm.eA6[5 * es + i] = w1.z;
    sm.eAl6[i] = l0.x; sm.eAl6[es + i] = l0.y; sm.eAl6[2 * es + i] = l0.z;
    sm.eAl6[3 * es + i] = l1.x; sm.eAl6[4 * es + i] = l1.y; sm.eAl6[5 * es + i] = l1.z;
  }
  for (int i = t0; i < ps.neB; i += ts) {
    const uint32_t e = a.edges[B.e_off + i];
    sm.eB[i] = e;
    const float4 u0 = a.verts[B.v_off + (e & 0xffffu)], u1 = a.verts[B.v_off + (e >> 16)];
    const V3 l0 = map_vertex(ps.kindB, u0.x, u0.y, u0.z, u0.w, ps.dB);
    const V3 l1 = map_vertex(ps.kindB, u1.x, u1.y, u1.z, u1.w, ps.dB);
    const int es = sm.es;
    sm.eB6[i] = l0.x; sm.eB6[es + i] = l0.y; sm.eB6[2 * es + i] = l0.z;
    sm.eB6[3 * es + i] = l1.x; sm.eB6[4 * es + i] = l1.y; sm.eB6[5 * es + i] = l1.z;
  }
  // hull planes pre-scaled by k = log2(e) / tau (see sdf_planes); superquadric
  // rows as packed
  const float kA = ps.kindA == kHull ? ps.k2 : 1.f, kB = ps.kindB == kHull ? ps.k2 : 1.f;
  for (int i = t0; i < ps.npA; i += ts) {
    const float4 q = a.planes[A.p_off + i];
    sm.pA[i] = make_float4(q.x * kA, q.y * kA, q.z * kA, q.w * kA);
  }
  for (int i = t0; i < ps.npB; i += ts) {
    const float4 q = a.planes[B.p_off + i];
    sm.pB[i] = make_float4(q.x * kB, q.y * kB, q.z * kB, q.w * kB);
  }
}

__device__ __forceinline__ void pair_stage(const FwdArgs& a, int pi, const PairShared& ps, const PairSmem& sm) {
  pair_stage_by(a, pi, ps, sm, threadIdx.x, blockDim.x);
}

// Next pair of this CTA: from the size-ordered work queue when one is given
// (largest pairs first, an atomic counter shared by all CTAs), else a static
// grid stride.  Called by every thread of the CTA.
__device__ __forceinline__ int next_pair(const FwdArgs& a, int& slot_iter) {
  if (a.work_counter) {
    __shared__ int next;
    __syncthreads();
    if (threadIdx.x == 0) next = atomicAdd(a.work_counter, 1);
    __syncthreads();
    int i = next;
    if (i >= a.n_pairs) return -1;
    return a.order ? a.order[i] : i;
  }
  int i = blockIdx.x + slot_iter * gridDim.x;
  ++slot_iter;
  if (i >= a.n_pairs) return -1;
  return a.order ? a.order[i] : i;
}

__device__ __forceinline__ V3 ld3(const float4& f) { return v3(f.x, f.y, f.z); }

struct PairBodies {
  Body A, B;
};

__device__ __forceinline__ PairBodies pair_bodies(const PairShared& ps, const PairSmem& sm) {
  PairBodies b;
  b.A.kind = ps.kindA; b.A.dims = ps.dA; b.A.planes = sm.pA; b.A.n_planes = ps.npA;
  b.B.kind = ps.kindB; b.B.dims = ps.dB; b.B.planes = sm.pB; b.B.n_planes = ps.npB;
  return b;
}

// SDF of A at a B-frame point: value and the gradient rotated into B's frame.
__device__ __forceinline__ Sdf sdfA_at(const PairShared& ps, const Body& A, V3 y) {
  V3 x = mulT(ps.Rrel, y - ps.trel);
  Sdf s = body_sdf(A, x, ps.tau, ps.inv_tau);
  s.g = mul(ps.Rrel, s.g);
  return s;
}
__device__ __forceinline__ Sdf sdfB_at(const PairShared& ps, const Body& B, V3 y) {
  return body_sdf(B, y, ps.tau, ps.inv_tau);
}

// Vertex-SDF candidate c in [0, nvA + nvB): A's vertices against B, then B's
// against A (Sec. IV-C).  Payload (p, d, n, w), score -w d.
__device__ __forceinline__ float vs_candidate(const PairShared& ps, const PairSmem& sm,
                                              const PairBodies& bb, int c, float (&y)[8]) {
  V3 p;
  Sdf s;
  if (c < ps.nvA) {
    p = ld3(sm.vA[c]);
    s = sdfB_at(ps, bb.B, p);
  } else {
    p = ld3(sm.vB[c - ps.nvA]);
    s = sdfA_at(ps, bb.A, p);
  }
  V3 n = normal_of(s.g, ps.tau);
  float w = sigmoid(-s.phi * ps.inv_tau);
  y[0] = p.x; y[1] = p.y; y[2] = p.z; y[3] = s.phi;
  y[4] = n.x; y[5] = n.y; y[6] = n.z; y[7] = w;
  return -w * s.phi;
}

// Edge endpoints of element (k, l) from the SoA endpoint arrays (lanes of a
// warp take consecutive l, so B's reads are conflict-free and A's broadcast).
struct EdgePair {
  V3 a0, a1, b0, b1;
  int k;
};
__device__ __forceinline__ EdgePair edge_pair(const PairSmem& sm, int k, int l) {
  const int es = sm.es;
  EdgePair e;
  e.k = k;
  e.a0 = v3(sm.eA6[k], sm.eA6[es + k], sm.eA6[2 * es + k]);
  e.a1 = v3(sm.eA6[3 * es + k], sm.eA6[4 * es + k], sm.eA6[5 * es + k]);
  e.b0 = v3(sm.eB6[l], sm.eB6[es + l], sm.eB6[2 * es + l]);
  e.b1 = v3(sm.eB6[3 * es + l], sm.eB6[4 * es + l], sm.eB6[5 * es + l]);
  return e;
}

// Witness points of an edge pair (Sec. IV-D2, IV-D3).
struct Witness {
  V3 e1, e2, delta;
  float dbar, con;
  QPOut qp;
};
__device__ __forceinline__ Witness ee_witness_from(const EdgePair& e, const QPOut& qp) {
  Witness w;
  w.qp = qp;
  w.e1 = fma3(w.qp.a1, e.a1 - e.a0, e.a0);
  w.e2 = fma3(w.qp.a2, e.b1 - e.b0, e.b0);
  w.delta = w.e1 - w.e2;
  float r2 = dot(w.delta, w.delta);
  w.dbar = sqrt_(r2);
  w.con = w.qp.con;
  return w;
}
__device__ __forceinline__ Witness ee_witness(const EdgePair& e, const Params& p) {
  QPPre q = qp_setup(e.a0, e.a1, e.b0, e.b1, p.w_reg);
  return ee_witness_from(e, qp_solve(q, p.w_reg, p));
}

// Both E-E candidates of element (k, l) (Sec. IV-D3): sign, penetration,
// nearest-neighbour (from the soft row / column minima L), clashing, activity.
// A's normal at its own witness is evaluated from A's local vertices: the SDF
// normal near a mesh corner turns at a rate ~1/tau, and a frame round trip of
// e1* would add FP32 position error that the soft sign then amplifies.
// kCls 1: A is a hull and B a box, capsule, cylinder or ellipsoid (compiled without
// the other kinds' branches); 0: any kinds.
template <int kCls = 0>
__device__ __forceinline__ void ee_candidates(const PairShared& ps, const PairSmem& sm,
                                              const PairBodies& bb, const EdgePair& ep,
                                              const Witness& w, float rowL, float colL,
                                              float (&y1)[8], float (&y2)[8], float& s1, float& s2) {
  const float tau = ps.tau, it = ps.inv_tau;
  const int es = sm.es, k = ep.k;
  const V3 la0 = v3(sm.eAl6[k], sm.eAl6[es + k], sm.eAl6[2 * es + k]);
  const V3 la1 = v3(sm.eAl6[3 * es + k], sm.eAl6[4 * es + k], sm.eAl6[5 * es + k]);
  V3 e1l = fma3(w.qp.a1, la1 - la0, la0);
  V3 e1 = w.e1, e2 = w.e2, delta = w.delta;
  float dbar = w.dbar;
  if (ps.trace) {  // witnesses onto their own body's SDF surface (e1* on A, e2* on B)
    e1l = trace_to_surface(bb.A, e1l, ps.trace, tau, it);
    e2 = trace_to_surface(bb.B, e2, ps.trace, tau, it);
    e1 = mul(ps.Rrel, e1l) + ps.trel;
    delta = e1 - e2;
    dbar = sqrt_(dot(delta, delta));
  }
  V3 nbar = delta * rsq(dot(delta, delta) + tau * tau);
  Sdf B_e1, B_e2, A_e2, A_e1;
  if (kCls == 1) {                                     // phi_B(e1*), nu_B(e2*)
    B_e1 = prim_sdf(bb.B, e1, tau, it);
    B_e2 = prim_sdf(bb.B, e2, tau, it);
  } else {
    body_sdf2(bb.B, e1, e2, tau, it, B_e1, B_e2);
  }
  const V3 x2 = mulT(ps.Rrel, e2 - ps.trel);
  // A hull's sums without a shift (sdf_planes_ee) while e1* is within a scaled
  // distance of 60 of A's edge (see sdf_planes_ee).
  float pen2 = -1.f, safe1 = 1.f;
  bool fast = false;
  if (!ps.trace && (kCls == 1 || bb.A.kind == kHull)) {
    const V3 t1 = la1 - la0;
    const float ex = fmaxf(fmaxf(-w.qp.a1, w.qp.a1 - 1.f), 0.f) * ps.k2;
    fast = ex * ex * dot(t1, t1) <= 3600.f;
  }
  if (fast) {
    float S1, S2;
    sdf_planes_ee(x2, e1l, bb.A.planes, bb.A.n_planes, tau, S1, S2, A_e1.g);
    pen2 = rcp(1.f + S1);
    safe1 = rcp(1.f + S2);
  } else {
    if (kCls == 1) sdf_planes2(x2, e1l, bb.A.planes, bb.A.n_planes, tau, A_e2, A_e1);
    else body_sdf2(bb.A, x2, e1l, tau, it, A_e2, A_e1);  // phi_A(e2*), nu_A(e1*) in A's frame
    pen2 = sigmoid(-A_e2.phi * it);
    safe1 = sigmoid(-A_e1.phi * it);
  }
  A_e1.g = mul(ps.Rrel, A_e1.g);
  V3 nuB = normal_of(B_e2.g, tau);
  V3 nuA = normal_of(A_e1.g, tau);
  float g1 = tanh_k(dot(nuB, nbar), ps.k2);
  float g2 = tanh_k(-dot(nuA, nbar), ps.k2);
  float pen1 = sigmoid_k(-B_e1.phi, ps.k2);
  float cl = sigmoid_k(-dot(nuA, nuB), ps.k2);
  float nn1 = ex2((rowL - w.dbar) * ps.k2);
  float nn2 = ex2((colL - w.dbar) * ps.k2);
  float base = w.con * cl;
  float w1 = base * pen1 * nn1, w2 = base * pen2 * nn2;
  if (ps.preselect) {  // safeguard: each witness inside its own body
    w1 *= safe1;
    w2 *= sigmoid(-B_e2.phi * it);
  }
  float d1 = g1 * dbar, d2 = g2 * dbar;
  y1[0] = e1.x; y1[1] = e1.y; y1[2] = e1.z; y1[3] = d1;
  y1[4] = g1 * nbar.x; y1[5] = g1 * nbar.y; y1[6] = g1 * nbar.z; y1[7] = w1;
  y2[0] = e2.x; y2[1] = e2.y; y2[2] = e2.z; y2[3] = d2;
  y2[4] = -g2 * nbar.x; y2[5] = -g2 * nbar.y; y2[6] = -g2 * nbar.z; y2[7] = w2;
  s1 = -w1 * d1;
  s2 = -w2 * d2;
}

// ---------------------------------------------------------------- soft pre-selection
// (Sec. IV-A; Supplement B).  Four selections per pair: A's vertices (kind 0),
// B's vertices (1), A's edges (2), B's edges (3).  An item's score is its depth
// -phi_other (vertices) or the mean of its corners' (edges); its payload is what
// the contacts use: positions in B's frame, A's local positions and the
// capsule-template cap signs (sel_width floats).
__host__ __device__ constexpr int sel_width(int kind) { return kind == 0 ? 7 : kind == 1 ? 4 : kind == 2 ? 14 : 8; }

struct SelArea {
  float* m[2];      // vertex depths of A and B (phi of the other body)
  float* item[4];   // kMaxSel x kSelPayload selected payloads per selection
  float* info[4];   // per selection: s^_k, Z_k, index of the k-th top item (bits)
};
__device__ __forceinline__ SelArea sel_area(const PairSmem& sm) {
  SelArea A;
  A.m[0] = sm.sel;
  A.m[1] = sm.sel + sm.vs;
  float* q = sm.sel + 2 * sm.vs;
  for (int j = 0; j < 4; ++j) {
    A.item[j] = q;
    q += kMaxSel * sel_width(j);
  }
  for (int j = 0; j < 4; ++j) {
    A.info[j] = q;
    q += 3 * kMaxSel;
  }
  return A;
}

__device__ __forceinline__ float sel_score(const PairSmem& sm, const SelArea& A, int kind, int i) {
  switch (kind) {
    case 0: return -A.m[0][i];
    case 1: return -A.m[1][i];
    case 2: { const uint32_t e = sm.eA[i]; return -0.5f * (A.m[0][e & 0xffffu] + A.m[0][e >> 16]); }
    default: { const uint32_t e = sm.eB[i]; return -0.5f * (A.m[1][e & 0xffffu] + A.m[1][e >> 16]); }
  }
}

template <int P>
__device__ __forceinline__ void sel_payload(const PairSmem& sm, int kind, int i, float (&v)[P]) {
  const int es = sm.es;
  if (kind == 0) {
    const float4 a = sm.vA[i], b = sm.vAl[i];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = b.x; v[4] = b.y; v[5] = b.z; v[6] = b.w;
  } else if (kind == 1) {
    const float4 a = sm.vB[i];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if (kind == 2) {
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = sm.eA6[c * es + i];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[6 + c] = sm.eAl6[c * es + i];
    const uint32_t e = sm.eA[i];
    v[12] = sm.vAl[e & 0xffffu].w;
    v[13] = sm.vAl[e >> 16].w;
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = sm.eB6[c * es + i];
    const uint32_t e = sm.eB[i];
    v[6] = sm.vB[e & 0xffffu].w;
    v[7] = sm.vB[e >> 16].w;
  }
}

// One warp per selection: the K largest scores by K arg-max passes in (score
// desc, index asc) order, then the SoftSort rows exp(-|s^_k - x_i| / tau) / Z_k
// applied to the items' payloads.  Records s^_k, Z_k and the k-th item's index.
template <int P>
__device__ __forceinline__ void warp_soft_select(int n, int K, float k2, int kind, const PairSmem& sm,
                                                 const SelArea& A) {
  const int lane = threadIdx.x & 31;
  float* dst = A.item[kind];
  float* info = A.info[kind];
  float prev_s = 3.0e38f;
  int prev_i = -1;
  for (int k = 0; k < K; ++k) {
    // the next item in (score desc, index asc) order after (prev_s, prev_i)
    float bs = -3.0e38f;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
      const float x = sel_score(sm, A, kind, i);
      const bool after = x < prev_s || (x == prev_s && i > prev_i);
      if (after && (x > bs || (x == bs && i < bi))) {
        bs = x;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(kFull, bs, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      if (os > bs || (os == bs && oi < bi)) {
        bs = os;
        bi = oi;
      }
    }
    prev_s = bs;
    prev_i = bi;
    // SoftSort row k
    float acc[P + 1];
#pragma unroll
    for (int c = 0; c <= P; ++c) acc[c] = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float e = ex2(-fabsf(bs - sel_score(sm, A, kind, i)) * k2);
      float v[P];
      sel_payload<P>(sm, kind, i, v);
      acc[0] += e;
#pragma unroll
      for (int c = 0; c < P; ++c) acc[1 + c] = fmaf(e, v[c], acc[1 + c]);
    }
#pragma unroll
    for (int c = 0; c <= P; ++c) acc[c] = warp_sum(acc[c]);
    if (lane == 0) {
      const float iz = 1.0f / acc[0];
#pragma unroll
      for (int c = 0; c < P; ++c) dst[k * P + c] = acc[1 + c] * iz;
      info[k] = bs;
      info[kMaxSel + k] = acc[0];
      info[2 * kMaxSel + k] = __int_as_float(bi);
    }
  }
}

// Cooperative: vertex depths, the four soft selections, and the selected items
// copied over the pair's staged vertices / edge endpoints (the original counts
// are kept in ps.n*0).  Contains __syncthreads: all threads must call.
__device__ inline void preselect_pair(const FwdArgs& a, PairShared& ps, const PairSmem& sm, const PairBodies& bb) {
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const SelArea A = sel_area(sm);
  for (int i = threadIdx.x; i < ps.nvA; i += blockDim.x) A.m[0][i] = sdfB_at(ps, bb.B, ld3(sm.vA[i])).phi;
  for (int i = threadIdx.x; i < ps.nvB; i += blockDim.x) A.m[1][i] = sdfA_at(ps, bb.A, ld3(sm.vB[i])).phi;
  __syncthreads();
  const int kvA = a.p.top_verts ? min(a.p.top_verts, ps.nvA) : 0;
  const int kvB = a.p.top_verts ? min(a.p.top_verts, ps.nvB) : 0;
  const int keA = a.p.top_edges ? min(a.p.top_edges, ps.neA) : 0;
  const int keB = a.p.top_edges ? min(a.p.top_edges, ps.neB) : 0;
  for (int job = warp; job < 4; job += nwarps) {
    if (job == 0 && kvA) warp_soft_select<7>(ps.nvA, kvA, ps.k2, 0, sm, A);
    if (job == 1 && kvB) warp_soft_select<4>(ps.nvB, kvB, ps.k2, 1, sm, A);
    if (job == 2 && keA) warp_soft_select<14>(ps.neA, keA, ps.k2, 2, sm, A);
    if (job == 3 && keB) warp_soft_select<8>(ps.neB, keB, ps.k2, 3, sm, A);
  }
  __syncthreads();
  const int es = sm.es;
  for (int i = threadIdx.x; i < kvA; i += blockDim.x) {
    const float* v = A.item[0] + 7 * i;
    sm.vA[i] = make_float4(v[0], v[1], v[2], 0.f);
    sm.vAl[i] = make_float4(v[3], v[4], v[5], v[6]);
  }
  for (int i = threadIdx.x; i < kvB; i += blockDim.x) {
    const float* v = A.item[1] + 4 * i;
    sm.vB[i] = make_float4(v[0], v[1], v[2], v[3]);
  }
  for (int i = threadIdx.x; i < keA; i += blockDim.x) {
    const float* v = A.item[2] + 14 * i;
    for (int c = 0; c < 6; ++c) {
      sm.eA6[c * es + i] = v[c];
      sm.eAl6[c * es + i] = v[6 + c];
    }
  }
  for (int i = threadIdx.x; i < keB; i += blockDim.x) {
    const float* v = A.item[3] + 8 * i;
    for (int c = 0; c < 6; ++c) sm.eB6[c * es + i] = v[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ps.nvA0 = ps.nvA; ps.nvB0 = ps.nvB; ps.neA0 = ps.neA; ps.neB0 = ps.neB;
    ps.kv[0] = kvA; ps.kv[1] = kvB; ps.kv[2] = keA; ps.kv[3] = keB;
    if (kvA) ps.nvA = kvA;
    if (kvB) ps.nvB = kvB;
    if (keA) ps.neA = keA;
    if (keB) ps.neB = keB;
  }
  __syncthreads();
}

}  // namespace cm
