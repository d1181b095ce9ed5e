// cm_order.cu -- size-bucketed work order of a batch of pairs.
//
// One CTA estimates every pair's arithmetic (vertex-SDF work plus E_A x E_B
// witness solves with four SDF evaluations each), buckets the estimates by
// powers of two and writes the pair indices bucket by bucket, largest first
// (for the adjoint, kind combination by kind combination).
// The manifold kernels then pull pairs from this list through an atomic
// counter, so the long pairs start first and the short ones fill the tail.
#include "cm_internal.h"

namespace cm {

__device__ __forceinline__ int planes_cost(const GeomHeader& g) {
  return g.kind == kBox ? 6 : (g.kind == kHull ? g.n_planes : 8);
}

// Bucket of pair i: the power of two of its estimated work, and with by_kind the
// pair's (kind of A, kind of B) as the major key, so that pairs of one kind
// combination run together (the adjoint's per-kind code then stays hot in the
// instruction cache).
constexpr int kKinds = 6, kSizeBuckets = 64, kBuckets = kKinds * kKinds * kSizeBuckets;
__device__ __forceinline__ int pair_bucket(const int32_t* pg, const GeomHeader* hdr, int n_geoms, int i,
                                           int by_kind) {
  const int ga = pg[2 * i], gb = pg[2 * i + 1];
  if (ga < 0 || ga >= n_geoms || gb < 0 || gb >= n_geoms) return 0;
  const GeomHeader& A = hdr[ga];
  const GeomHeader& B = hdr[gb];
  const long long fA = planes_cost(A), fB = planes_cost(B);
  const long long c = (long long)A.n_verts * (fB + 4) + (long long)B.n_verts * (fA + 4) +
                      (long long)A.n_edges * B.n_edges * (60 + 2 * fA + 2 * fB);
  const int b = 63 - __clzll(c > 1 ? c : 1);
  return by_kind ? (A.kind * kKinds + B.kind) * kSizeBuckets + b : b;
}

__global__ void __launch_bounds__(1024) cm_order_kernel(const int32_t* pg, const GeomHeader* hdr, int n_geoms, int n,
                                                        int32_t* order, int32_t* counter, int by_kind) {
  __shared__ int hist[kBuckets], off[kBuckets];
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[b] = 0;
  if (threadIdx.x == 0) *counter = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[pair_bucket(pg, hdr, n_geoms, i, by_kind)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {  // kind combinations in turn, each largest work first
    int acc = 0;
    for (int g = 0; g < kKinds * kKinds; ++g)
      for (int b = kSizeBuckets - 1; b >= 0; --b) {
        off[g * kSizeBuckets + b] = acc;
        acc += hist[g * kSizeBuckets + b];
      }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int pos = atomicAdd(&off[pair_bucket(pg, hdr, n_geoms, i, by_kind)], 1);
    order[pos] = i;
  }
}

cudaError_t launch_order(const int32_t* pair_geoms, const GeomHeader* hdr, int n_geoms, int n, int32_t* order,
                         int32_t* counter, int by_kind, cudaStream_t s) {
  cm_order_kernel<<<1, 1024, 0, s>>>(pair_geoms, hdr, n_geoms, n, order, counter, by_kind);
  return cudaGetLastError();
}

}  // namespace cm
