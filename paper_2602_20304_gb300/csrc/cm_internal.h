// cm_internal.h -- structures shared by the host runtime and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cm_math.cuh"

namespace cm {

// One registered geometry inside the packed device store.
struct GeomHeader {
  int32_t kind;
  int32_t n_verts, n_edges, n_planes;
  int32_t v_off, e_off, p_off;  // offsets into verts (float4), edges (uint32), planes (float4)
  int32_t pad0;
  float dims[3];
  float pad1;
};
static_assert(sizeof(GeomHeader) == 48, "GeomHeader layout");

// Byte offsets of the per-CTA shared-memory carve-up (sized on the host from the
// largest registered geometry).
struct SmemLayout {
  int vA, vAl, vB, pA, pB, eA, eB, rowL, colL, warp, eA6, eAl6, eB6, sel, sadj;
  int total;
  int max_v, max_e, max_p;
};

struct FwdArgs {
  const GeomHeader* hdr;
  int32_t n_geoms;
  const float4* verts;
  const uint32_t* edges;  // (i | j << 16)
  const float4* planes;
  int32_t n_pairs;
  const int32_t* pair_geoms;
  const float* poses;
  const float* dims;  // may be null
  const float* tau;   // may be null
  Params p;
  float* out;
  float* scratch;            // per-CTA slices of scratch_stride floats (E-E distances)
  int64_t scratch_stride;
  int* err;                  // sticky device error: first bad pair index + 1
  SmemLayout sm;
  int32_t* work_counter;     // persistent-CTA work queue (may be null: static striding)
  int32_t store_alpha;       // pass 1 keeps (alpha1, alpha2, con) beside dbar: 4 scratch floats per edge pair
  const int32_t* order;      // optional pair order for the work queue (may be null)
  // Per-pair forward record (may be null): written by the forward, read by the
  // adjoint, saved_stride floats per pair (see kRecHead).
  float* saved;
  int64_t saved_stride;
  int32_t saved_first;  // the forward writes records of pairs >= saved_first, from record 0
  // Candidate dump (may be null): every candidate of pair i as 8 floats (p, d, n, w in
  // world coordinates) at row dump_off[i] + its id, for rows below dump_rows.
  float* dump;
  const int64_t* dump_off;
  int64_t dump_rows;
};

// Optional outputs of one step beside the manifold (see FwdArgs).
struct StepExtras {
  float* saved = nullptr;
  int64_t saved_stride = 0;
  int32_t saved_first = 0;
  float* dump = nullptr;
  const int64_t* dump_off = nullptr;
  int64_t dump_rows = 0;
};

// Forward record of one pair, as the adjoint reads it: the K selected scores s^_k,
// their candidate ids (int bits), the SoftSort normalisers Z_k and the K output rows
// in B's frame (8 floats each) -- kRecHead * K floats -- then the soft row minima of
// the E-E distance matrix (max_e slots) and its soft column minima (max_e slots).
constexpr int kRecHead = 11;
// Adjoint scratch per edge pair: the distance, t1, t2, the QP result (3) and its
// adjoints (3), as arrays of scratch_stride floats in each CTA's slice.
constexpr int kBwdScratchArrays = 9;

// Launch shape of a manifold kernel: threads per CTA, CTAs per SM (0 = as many
// as fit) and whether pairs are pulled from the size-ordered work list.
struct LaunchCfg {
  int block;
  int per_sm;
  int ordered;
  int warp = 0;  // forward only: one warp per pair (cm_fwd_warp_kernel)
};

constexpr int kMaxK = 16;
constexpr int kMaxSel = 32;  // soft pre-selected items per body (CM_MAX_SELECT)
constexpr int kSqRows = 5;   // device float4 rows per superquadric of an SQ_UNION
// Pre-selection staging: vertex depths of both bodies (2 max_v) + the four soft
// selections' payloads (7, 4, 14 and 8 floats per item: positions in B's frame,
// A's local positions, capsule cap signs) and per selection s^_k, Z_k and the
// index of the k-th top item.
constexpr int kSelFloats = kMaxSel * (7 + 4 + 14 + 8) + 4 * 3 * kMaxSel;
// Adjoint of a pre-selection: local-frame adjoints of the selected items
// (3 + 3 + 6 + 6 floats) and the vertex-depth adjoints of both bodies (2 max_v).
constexpr int kSelAdjFloats = kMaxSel * (3 + 3 + 6 + 6);
// Per-warp SoftSort area: kMaxK payload slots of 8 floats, the list's scores, ids
// and slots, C (9), the K-th score and C's reference (see cm_softsort.cuh).
constexpr int kWarpStateFloats = 188;

// Raises `kernel`'s dynamic shared-memory limit to `bytes` on the current device,
// once per (kernel, device): the attribute belongs to the device's context, so a
// process that uses several GPUs sets it on each.  Occupancy queries above 48 KB
// and launches call it first.
cudaError_t ensure_smem_attr(const void* kernel, int bytes);

cudaError_t launch_fwd(const FwdArgs& a, int grid, int block, cudaStream_t s);
int fwd_max_blocks_per_sm(int block, int smem_bytes);
// One warp per pair (cm_fwd_warp.cu): a.sm is the single-warp layout without the
// pre-selection area; each warp's slice adds 4 max_e^2 floats of edge-pair data.
cudaError_t launch_fwd_warp(const FwdArgs& a, int grid, int block, cudaStream_t s);
int fwd_warp_bytes(const SmemLayout& L);
int fwd_warp_max_blocks_per_sm(int block, int smem_bytes);
bool fwd_warp_fits(const SmemLayout& L, int block);
cudaError_t launch_bwd(const FwdArgs& a, const float* grad_out, float* grad_poses, float* grad_dims, int grid,
                       int block, int per_sm, cudaStream_t s);
int bwd_max_blocks_per_sm(int block, int smem_bytes, int per_sm);
cudaError_t launch_order(const int32_t* pair_geoms, const GeomHeader* hdr, int n_geoms, int n, int32_t* order,
                         int32_t* counter, int by_kind, cudaStream_t s);

}  // namespace cm
