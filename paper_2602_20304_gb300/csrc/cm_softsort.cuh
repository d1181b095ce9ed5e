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
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
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

// Folds another warp's stored state (its area) into this warp's state.
__device__ __forceinline__ void wtk_merge(WarpTopK& st, const float* src, int K, float k2) {
  const int lane = threadIdx.x & 31;
  float y[8];
  float s = kNegInf;
  bool valid = false;
  int id = -1;
  if (lane < K) {
    s = src[kSsScore + lane];
    valid = s != kNegInf;
    id = __float_as_int(src[kSsId + lane]);
    const float* ys = src + kSsSlots + 8 * __float_as_int(src[kSsSlot + lane]);
#pragma unroll
    for (int c = 0; c < 8; ++c) y[c] = valid ? ys[c] : 0.f;
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) y[c] = 0.f;
  }
  wtk_push(st, valid, s, y, K, k2, id);
  const float ref_w = src[kSsRef];
  if (ref_w != kNegInf) {
    // both references lie at or below this warp's K-th score now: take the larger
    // and scale both accumulators down to it
    const float r = fmaxf(st.ref, ref_w);
    const float fo = st.ref == kNegInf ? 0.f : ex2((st.ref - r) * k2);
#pragma unroll
    for (int c = 0; c < 9; ++c) st.C[c] *= fo;
    if (lane == 0) {
      const float fw = ex2((ref_w - r) * k2);
#pragma unroll
      for (int c = 0; c < 9; ++c) st.C[c] = fmaf(fw, src[kSsC + c], st.C[c]);
    }
    st.ref = r;
  }
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
