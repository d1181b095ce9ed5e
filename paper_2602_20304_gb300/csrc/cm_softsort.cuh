// cm_softsort.cuh -- streaming SoftSort top-K reduction, one warp per stream.
//
// SoftSort (Sec. III): with s^_1 >= ... >= s^_K the K largest scores,
//   out_k = sum_i G_ki y_i / sum_i G_ki,   G_ki = exp(-|s^_k - s_i| / tau).
// All candidates below the K-th largest score s^_K contribute to every row
// through exp((s_i - s^_K)/tau) * exp((s^_K - s^_k)/tau), so one accumulator
//   C = sum_{i not in top-K} exp((s_i - s^_K)/tau) (1, y_i)
// and the K top entries themselves determine all K rows:
//   out_k ~ sum_{j<=K} exp(-|s^_k - s^_j|/tau) (1, y_j) + exp((s^_K - s^_k)/tau) C.
// The warp keeps the sorted top-K list distributed over lanes 0..K-1 and each
// lane its own share of C relative to the warp-uniform threshold s^_K.  A new
// candidate above the threshold is inserted (rare after the list warms up);
// the evicted entry joins C and C is rescaled by exp((old - new)/tau) <= 1.
// Every factor applied is <= 1, so nothing overflows and nothing cancels.
#pragma once

#include "cm_math.cuh"

namespace cm {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kNegInf = -INFINITY;

struct WarpTopK {
  float ls;      // score of the list entry held by this lane (lanes < K), -inf if empty
  float ly[8];   // its payload (p, d, n, w)
  int lid;       // its candidate id
  float C[9];    // this lane's share of the below-threshold accumulator (weight, payload)
  float thr;     // warp-uniform K-th largest score so far (-inf until K entries)
};

__device__ __forceinline__ void wtk_init(WarpTopK& st) {
  st.ls = kNegInf;
  st.lid = -1;
#pragma unroll
  for (int c = 0; c < 8; ++c) st.ly[c] = 0.f;
#pragma unroll
  for (int c = 0; c < 9; ++c) st.C[c] = 0.f;
  st.thr = kNegInf;
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
    float yn[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) yn[c] = __shfl_sync(kFull, y[c], src);
    const int pos = __popc(__ballot_sync(kFull, lane < K && st.ls >= sn));
    const float ev_s = __shfl_sync(kFull, st.ls, K - 1);
    float old_y[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) old_y[c] = st.ly[c];
    const float up_s = __shfl_up_sync(kFull, st.ls, 1);
    const int up_id = __shfl_up_sync(kFull, st.lid, 1);
    float up_y[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) up_y[c] = __shfl_up_sync(kFull, st.ly[c], 1);
    if (lane < K) {
      if (lane > pos) {
        st.ls = up_s;
        st.lid = up_id;
#pragma unroll
        for (int c = 0; c < 8; ++c) st.ly[c] = up_y[c];
      } else if (lane == pos) {
        st.ls = sn;
        st.lid = idn;
#pragma unroll
        for (int c = 0; c < 8; ++c) st.ly[c] = yn[c];
      }
    }
    const float new_thr = __shfl_sync(kFull, st.ls, K - 1);
    if (new_thr != kNegInf) {
      const float f = (st.thr == kNegInf) ? 0.f : ex2((st.thr - new_thr) * k2);
#pragma unroll
      for (int c = 0; c < 9; ++c) st.C[c] *= f;
      if (lane == K - 1 && ev_s != kNegInf) {
        // the evicted entry scored exactly the old threshold: its weight is f
        st.C[0] += f;
#pragma unroll
        for (int c = 0; c < 8; ++c) st.C[1 + c] = fmaf(f, old_y[c], st.C[1 + c]);
      }
      st.thr = new_thr;
    }
    if (lane == src) valid = false;
    m = __ballot_sync(kFull, valid && s > st.thr);
  }
  if (valid) {
    const float e = ex2((s - st.thr) * k2);
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

// Writes a warp's state to shared memory: K list entries (score + 8), the
// warp-summed C (9) and the threshold.
__device__ __forceinline__ void wtk_store(const WarpTopK& st, float* dst, int K) {
  const int lane = threadIdx.x & 31;
  if (lane < K) {
    dst[lane * 9] = st.ls;
#pragma unroll
    for (int c = 0; c < 8; ++c) dst[lane * 9 + 1 + c] = st.ly[c];
  }
  float Cs[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) Cs[c] = warp_sum(st.C[c]);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) dst[16 * 9 + c] = Cs[c];
    dst[16 * 9 + 9] = st.thr;
  }
  if (lane < K) dst[16 * 9 + 10 + lane] = __int_as_float(st.lid);
}

// Folds a stored warp state into this warp's state.
__device__ __forceinline__ void wtk_merge(WarpTopK& st, const float* src, int K, float k2) {
  const int lane = threadIdx.x & 31;
  float y[8];
  float s = kNegInf;
  bool valid = false;
  int id = -1;
  if (lane < K) {
    s = src[lane * 9];
    valid = s != kNegInf;
    id = __float_as_int(src[16 * 9 + 10 + lane]);
#pragma unroll
    for (int c = 0; c < 8; ++c) y[c] = src[lane * 9 + 1 + c];
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) y[c] = 0.f;
  }
  wtk_push(st, valid, s, y, K, k2, id);
  const float thr_w = src[16 * 9 + 9];
  if (lane == 0 && thr_w != kNegInf) {
    // thr_w <= st.thr once the other warp's K entries have been offered
    const float f = ex2((thr_w - st.thr) * k2);
#pragma unroll
    for (int c = 0; c < 9; ++c) st.C[c] = fmaf(f, src[16 * 9 + c], st.C[c]);
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
  const float fc = (lane < K) ? ex2((st.thr - sk) * k2) : 0.f;
#pragma unroll
  for (int c = 0; c < 9; ++c) num[c] = fc * Ct[c];
  for (int j = 0; j < K; ++j) {
    const float sj = __shfl_sync(kFull, st.ls, j);
    const float e = ex2(-fabsf(sk - sj) * k2);
    num[0] += e;
#pragma unroll
    for (int c = 0; c < 8; ++c) num[1 + c] = fmaf(e, __shfl_sync(kFull, st.ly[c], j), num[1 + c]);
  }
  const float inv = 1.0f / num[0];
#pragma unroll
  for (int c = 0; c < 8; ++c) y[c] = num[1 + c] * inv;
  if (Z) *Z = num[0];
}

}  // namespace cm
