// cm_softsort.cuh -- streaming SoftSort top-K reduction, one warp per stream.
//
// SoftSort (Sec. III): with s^_1 >= ... >= s^_K the K largest scores,
//   out_k = sum_i G_ki y_i / sum_i G_ki,   G_ki = exp(-|s^_k - s_i| / tau).
// All candidates below the K-th largest score s^_K contribute to every row
// through exp((s_i - r)/tau) * exp((r - s^_k)/tau) for any reference r, so one
// accumulator
//   C = sum_{i not in top-K} exp((s_i - r)/tau) (1, y_i)
// and the K top entries themselves determine all K rows:
//   out_k ~ sum_{j<=K} exp(-|s^_k - s^_j|/tau) (1, y_j) + exp((r - s^_k)/tau) C.
// The warp keeps the sorted top-K list distributed over lanes 0..K-1 (score,
// candidate id and the shared-memory slot holding the entry's payload) and
// each lane its own share of C.  The reference r is the K-th score at the time
// the list first filled up and is moved up to the current K-th score only when
// the two drift more than 64 / log2(e/tau) apart, so an insertion does not
// rescale C: every term added is <= 2^64 and nothing cancels.  A new candidate
// above the K-th score is inserted (rare after the list warms up); the evicted
// entry's payload is read back from its slot into C and the slot is reused.
#pragma once

#include "cm_math.cuh"

namespace cm {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kNegInf = -INFINITY;
constexpr float kRebase = 64.f;  // largest base-2 exponent of a term of C before the reference moves

// Per-warp shared-memory area of a stream (floats): payload slots (kMaxK x 8),
// then, written by wtk_store for a merge: scores, ids, slots of the list
// positions (kMaxK each), the warp-summed C (9), the K-th score and C's reference.
constexpr int kSsSlots = 0, kSsScore = 16 * 8, kSsId = kSsScore + 16, kSsSlot = kSsId + 16, kSsC = kSsSlot + 16,
              kSsThr = kSsC + 9, kSsRef = kSsThr + 1, kSsFloats = kSsRef + 1;

struct WarpTopK {
  float ls;      // score of the list entry held by this lane (lanes < K), -inf if empty
  int lid;       // its candidate id
  int lslot;     // its payload slot
  float C[9];    // this lane's share of the below-threshold accumulator (weight, payload), relative to ref
  float thr;     // warp-uniform K-th largest score so far (-inf until K entries)
  float ref;     // warp-uniform reference of C (-inf until K entries)
  int cnt;       // warp-uniform number of list entries
  float* area;   // this warp's shared-memory area (kSsFloats floats)
};

__device__ __forceinline__ void wtk_init(WarpTopK& st, float* area) {
  st.ls = kNegInf;
  st.lid = -1;
  st.lslot = 0;
#pragma unroll
  for (int c = 0; c < 9; ++c) st.C[c] = 0.f;
  st.thr = kNegInf;
  st.ref = kNegInf;
  st.cnt = 0;
  st.area = area;
}

// Moves C's reference up to the current K-th score once they drift apart (warp-uniform).
__device__ __forceinline__ void wtk_rebase(WarpTopK& st, float k2) {
  if ((st.thr - st.ref) * k2 > kRebase) {
    const float f = ex2((st.ref - st.thr) * k2);
#pragma unroll
    for (int c = 0; c < 9; ++c) st.C[c] *= f;
    st.ref = st.thr;
  }
}

// Offers one candidate per lane (valid lanes only).  All 32 lanes must call.
// k2 = log2(e) / tau.
__device__ __forceinline__ void wtk_push(WarpTopK& st, bool valid, float s, const float (&y)[8],
                                         int K, float k2, int id = -1) {
  const int lane = threadIdx.x & 31;
  unsigned m = __ballot_sync(kFull, valid && s > st.thr);
  while (m) {
    const int src = __ffs(m) - 1;
    const float sn = __shfl_sync(kFull, s, src);
    const int idn = __shfl_sync(kFull, id, src);
    const int pos = __popc(__ballot_sync(kFull, lane < K && st.ls >= sn));
    int slot = st.cnt;
    if (st.cnt == K) {  // the K-th entry leaves the list for C; its slot takes the new payload
      const float ev_s = __shfl_sync(kFull, st.ls, K - 1);
      slot = __shfl_sync(kFull, st.lslot, K - 1);
      if (lane == K - 1) {
        const float e = ex2((ev_s - st.ref) * k2);
        const float* ys = st.area + kSsSlots + 8 * slot;
        st.C[0] += e;
#pragma unroll
        for (int c = 0; c < 8; ++c) st.C[1 + c] = fmaf(e, ys[c], st.C[1 + c]);
      }
      __syncwarp();
    }
    if (lane == src) {
      float* yd = st.area + kSsSlots + 8 * slot;
#pragma unroll
      for (int c = 0; c < 8; ++c) yd[c] = y[c];
      valid = false;
    }
    const float up_s = __shfl_up_sync(kFull, st.ls, 1);
    const int up_id = __shfl_up_sync(kFull, st.lid, 1);
    const int up_slot = __shfl_up_sync(kFull, st.lslot, 1);
    if (lane < K) {
      if (lane > pos) {
        st.ls = up_s;
        st.lid = up_id;
        st.lslot = up_slot;
      } else if (lane == pos) {
        st.ls = sn;
        st.lid = idn;
        st.lslot = slot;
      }
    }
    st.cnt = min(st.cnt + 1, K);
    if (st.cnt == K) {
      st.thr = __shfl_sync(kFull, st.ls, K - 1);
      if (st.ref == kNegInf) st.ref = st.thr;
      wtk_rebase(st, k2);
    }
    __syncwarp();
    m = __ballot_sync(kFull, valid && s > st.thr);
  }
  if (valid) {  // below the K-th score (the list is full, ref is finite)
    const float e = ex2((s - st.ref) * k2);
    st.C[0] += e;
#pragma unroll
    for (int c = 0; c < 8; ++c) st.C[1 + c] = fmaf(e, y[c], st.C[1 + c]);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Writes the list (scores, ids, slots; the payloads already sit in the area's
// slots), the warp-summed C, the K-th score and C's reference into the warp's area.
__device__ __forceinline__ void wtk_store(const WarpTopK& st, int K) {
  const int lane = threadIdx.x & 31;
  float* dst = st.area;
  if (lane < K) {
    dst[kSsScore + lane] = st.ls;
    dst[kSsId + lane] = __int_as_float(st.lid);
    dst[kSsSlot + lane] = __int_as_float(st.lslot);
  }
  float Cs[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) Cs[c] = warp_sum(st.C[c]);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) dst[kSsC + c] = Cs[c];
    dst[kSsThr] = st.thr;
    dst[kSsRef] = st.ref;
  }
}

// Folds another warp's stored state (its area) into this warp's state in one
// parallel step: lanes 0..K-1 hold this warp's entries, lanes K..2K-1 the other
// warp's; each computes its rank among the 2K (score descending, this warp's
// entries first on ties, list order within a list), the first K stay, the rest
// join C.  The other warp's survivors move their payloads into this warp's
// slots freed by its evicted entries (or unused when its list was not full).
__device__ __forceinline__ void wtk_merge(WarpTopK& st, const float* src, int K, float k2) {
  const int lane = threadIdx.x & 31;
  const bool own = lane < K, other = lane >= K && lane < 2 * K;
  float cs = kNegInf;
  int cid = -1, cslot = 0;
  if (own) {
    cs = st.ls;
    cid = st.lid;
    cslot = st.lslot;
  } else if (other) {
    cs = src[kSsScore + lane - K];
    cid = __float_as_int(src[kSsId + lane - K]);
    cslot = __float_as_int(src[kSsSlot + lane - K]);
  }
  const bool valid = cs != kNegInf;
  int rank = 0;
  for (int j = 0; j < 2 * K; ++j) {
    const float sj = __shfl_sync(kFull, cs, j);
    rank += (sj > cs || (sj == cs && j < lane)) ? 1 : 0;
  }
  const bool keep = valid && rank < K, evict = valid && rank >= K;
  const int nvalid = __popc(__ballot_sync(kFull, valid));
  const int cnt = min(nvalid, K);
  const unsigned kth = __ballot_sync(kFull, keep && rank == K - 1);
  const float thr = cnt == K ? __shfl_sync(kFull, cs, __ffs(kth) - 1) : kNegInf;
  // C's new reference: the larger of the two (both at or below the new K-th score)
  const float ref_w = src[kSsRef];
  float r = fmaxf(st.ref, ref_w);
  if (r == kNegInf && cnt == K) r = thr;
  const float fo = st.ref == kNegInf ? 0.f : ex2((st.ref - r) * k2);
#pragma unroll
  for (int c = 0; c < 9; ++c) st.C[c] *= fo;
  if (lane == 0 && ref_w != kNegInf) {
    const float fw = ex2((ref_w - r) * k2);
#pragma unroll
    for (int c = 0; c < 9; ++c) st.C[c] = fmaf(fw, src[kSsC + c], st.C[c]);
  }
  if (evict) {  // evicted entries join C (r is finite: the merged list is full)
    const float e = ex2((cs - r) * k2);
    const float* ys = (own ? st.area : src) + kSsSlots + 8 * cslot;
    st.C[0] += e;
#pragma unroll
    for (int c = 0; c < 8; ++c) st.C[1 + c] = fmaf(e, ys[c], st.C[1 + c]);
  }
  __syncwarp();
  // the m-th surviving entry of the other warp takes the m-th freed slot of this one
  const unsigned lt = (1u << lane) - 1u;
  const unsigned ev_own = __ballot_sync(kFull, evict && own);
  const int own_cnt = __popc(__ballot_sync(kFull, own && valid));
  const int m = __popc(__ballot_sync(kFull, keep && other) & lt);
  const int nev = __popc(ev_own);
  int from = 0;
  if (keep && other && m < nev) {  // lane of the m-th evicted entry of this warp
    unsigned mm = ev_own;
    for (int t = 0; t < m; ++t) mm &= mm - 1u;
    from = __ffs(mm) - 1;
  }
  const int freed = __shfl_sync(kFull, cslot, from);
  if (keep && other) {
    const int slot = m < nev ? freed : own_cnt + (m - nev);
    const float* ys = src + kSsSlots + 8 * cslot;
    float* yd = st.area + kSsSlots + 8 * slot;
#pragma unroll
    for (int c = 0; c < 8; ++c) yd[c] = ys[c];
    cslot = slot;
  }
  // the kept entries take list positions = their ranks (this warp's store area as scratch)
  if (keep) {
    st.area[kSsScore + rank] = cs;
    st.area[kSsId + rank] = __int_as_float(cid);
    st.area[kSsSlot + rank] = __int_as_float(cslot);
  }
  __syncwarp();
  if (lane < K) {
    const bool has = lane < cnt;
    st.ls = has ? st.area[kSsScore + lane] : kNegInf;
    st.lid = has ? __float_as_int(st.area[kSsId + lane]) : -1;
    st.lslot = has ? __float_as_int(st.area[kSsSlot + lane]) : 0;
  }
  __syncwarp();
  st.cnt = cnt;
  st.thr = thr;
  st.ref = cnt == K ? r : kNegInf;
  if (cnt == K) wtk_rebase(st, k2);
}

// Final rows: lane k < K returns out_k in y (weights normalised) and, in Z, the
// row's normaliser sum_i exp(-|s^_k - s_i| / tau).  All lanes call.
__device__ __forceinline__ void wtk_finish(const WarpTopK& st, int K, float k2, float (&y)[8], float* Z = nullptr) {
  const int lane = threadIdx.x & 31;
  float Ct[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) Ct[c] = warp_sum(st.C[c]);
  const float sk = st.ls;
  float num[9];
  const float fc = (lane < K && st.ref != kNegInf) ? ex2((st.ref - sk) * k2) : 0.f;
#pragma unroll
  for (int c = 0; c < 9; ++c) num[c] = fc * Ct[c];
  for (int j = 0; j < K; ++j) {
    const float sj = __shfl_sync(kFull, st.ls, j);
    const int slot = __shfl_sync(kFull, st.lslot, j);
    const float* ys = st.area + kSsSlots + 8 * slot;
    const float e = ex2(-fabsf(sk - sj) * k2);
    num[0] += e;
#pragma unroll
    for (int c = 0; c < 8; ++c) num[1 + c] = fmaf(e, ys[c], num[1 + c]);
  }
  const float inv = 1.0f / num[0];
#pragma unroll
  for (int c = 0; c < 8; ++c) y[c] = num[1 + c] * inv;
  if (Z) *Z = num[0];
}

}  // namespace cm
