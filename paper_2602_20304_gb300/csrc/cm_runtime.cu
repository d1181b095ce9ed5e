// cm_runtime.cu -- host side of the C ABI declared in include/contact_manifold.h:
// context, packed geometry store, argument validation, scratch management and
// kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "contact_manifold.h"
#include "cm_context.h"

using namespace cm;

namespace cm {
namespace rt {
thread_local std::string g_last_error;

cm_status fail(cm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
cm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
namespace {
int align16(int x) { return (x + 15) & ~15; }
}  // namespace
}  // namespace rt
}  // namespace cm

using namespace cm::rt;



namespace cm {

cudaError_t ensure_smem_attr(const void* kernel, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> bytes set
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({kernel, dev});
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[{kernel, dev}] = bytes;
  return e;
}

namespace rt {

template <class T>
cudaError_t grow_upload(T*& dptr, size_t& cap, const std::vector<T>& host) {
  size_t n = std::max<size_t>(host.size(), 1);
  if (n > cap) {
    if (dptr) cudaFree(dptr);
    dptr = nullptr;
    size_t ncap = std::max(n, cap * 2);
    cudaError_t e = cudaMalloc(&dptr, ncap * sizeof(T));
    if (e != cudaSuccess) {
      cap = 0;
      return e;
    }
    cap = ncap;
  }
  if (!host.empty()) return cudaMemcpy(dptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
  return cudaSuccess;
}

cm_status sync_geometry_locked(cm_context* c) {
  if (c->device < 0) return fail(CM_ERR_INVALID_ARG, "host-only context: no device work");
  if (!c->dirty) return CM_OK;
  cudaError_t e;
  if ((e = grow_upload(c->d_hdr, c->cap_hdr, c->hdr)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  if ((e = grow_upload(c->d_verts, c->cap_verts, c->verts)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  if ((e = grow_upload(c->d_edges, c->cap_edges, c->edges)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  if ((e = grow_upload(c->d_planes, c->cap_planes, c->planes)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  c->dirty = false;
  ++c->geom_gen;
  return CM_OK;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

cm_status check_params(const cm_params* p) {
  if (!p) return fail(CM_ERR_INVALID_ARG, "params is NULL");
  if (!finite_pos(p->tau) || !finite_pos(p->eps_clip) || !finite_pos(p->eps_min) || !finite_pos(p->eps_comp))
    return fail(CM_ERR_INVALID_ARG, "tau and eps_* must be finite and > 0");
  if (!(std::isfinite(p->w_reg) && p->w_reg > 0.f))
    return fail(CM_ERR_INVALID_ARG, "w_reg must be finite and > 0 (the E-E QP needs it to be strictly convex)");
  if (p->K < 1 || p->K > CM_MAX_K) return fail(CM_ERR_INVALID_ARG, "K must be in 1..16");
  if (p->flags & ~7) return fail(CM_ERR_INVALID_ARG, "unknown flag bits");
  if (p->top_verts < 0 || p->top_verts > CM_MAX_SELECT || p->top_edges < 0 || p->top_edges > CM_MAX_SELECT)
    return fail(CM_ERR_INVALID_ARG, "top_verts and top_edges must be in 0..32");
  if (p->trace_iters < 0 || p->trace_iters > CM_MAX_TRACE)
    return fail(CM_ERR_INVALID_ARG, "trace_iters must be in 0..8");
  return CM_OK;
}

SmemLayout make_layout(const cm_context* c, int nwarps, int bwd, bool with_sel = true) {
  SmemLayout L;
  int o = 0;
  L.max_v = c->max_v;
  L.max_e = c->max_e;
  L.max_p = c->max_p;
  L.vA = o; o = align16(o + 16 * c->max_v);
  L.vAl = o; o = align16(o + 16 * c->max_v);
  L.vB = o; o = align16(o + 16 * c->max_v);
  L.pA = o; o = align16(o + 16 * c->max_p);
  L.pB = o; o = align16(o + 16 * c->max_p);
  L.eA = o; o = align16(o + 4 * c->max_e);
  L.eB = o; o = align16(o + 4 * c->max_e);
  L.rowL = o; o = align16(o + 8 * c->max_e);   // soft minima (+ row adjoint sums in the backward)
  L.colL = o; o = align16(o + 8 * c->max_e);
  L.warp = o; o = align16(o + 4 * kWarpStateFloats * nwarps);
  L.eA6 = o; o = align16(o + 24 * c->max_e);
  L.eAl6 = o; o = align16(o + 24 * c->max_e);
  L.eB6 = o; o = align16(o + 24 * c->max_e);
  L.sel = o;
  if (with_sel) o = align16(o + 4 * (2 * c->max_v + kSelFloats));
  L.sadj = o;
  if (bwd) o = align16(o + 4 * (kSelAdjFloats + 2 * c->max_v));  // pre-selection adjoint slots
  L.total = o;
  return L;
}

cm_status ensure_scratch(cm_context* c, size_t floats) {
  if (floats <= c->scratch_floats) return CM_OK;
  if (c->d_scratch) cudaFree(c->d_scratch);
  c->d_scratch = nullptr;
  c->scratch_floats = 0;
  cudaError_t e = cudaMalloc(&c->d_scratch, floats * sizeof(float));
  if (e != cudaSuccess) return fail(CM_ERR_OOM, std::string("scratch allocation: ") + cudaGetErrorString(e));
  c->scratch_floats = floats;
  return CM_OK;
}


cm_status ensure_order(cm_context* c, size_t n) {
  if (!c->d_counter) {
    cudaError_t e = cudaMalloc(&c->d_counter, sizeof(int32_t));
    if (e != cudaSuccess) return fail(CM_ERR_OOM, std::string("work counter allocation: ") + cudaGetErrorString(e));
  }
  if (n <= c->cap_order) return CM_OK;
  if (c->d_order) cudaFree(c->d_order);
  c->d_order = nullptr;
  c->cap_order = 0;
  cudaError_t e = cudaMalloc(&c->d_order, n * sizeof(int32_t));
  if (e != cudaSuccess) return fail(CM_ERR_OOM, std::string("work list allocation: ") + cudaGetErrorString(e));
  c->cap_order = n;
  return CM_OK;
}

cm_status check_k(const cm_context* c, const cm_params* params) {
  if (params->flags & CM_FLAG_HARD)
    return fail(CM_ERR_INVALID_ARG, "CM_FLAG_HARD applies to the witness-point routines only");
  if (params->flags & (CM_FLAG_NO_EE | CM_FLAG_ONE_SIDED)) {
    const int nv = params->top_verts ? std::min(params->top_verts, c->min_v) : c->min_v;
    const int min_cands = (params->flags & CM_FLAG_ONE_SIDED) ? nv : 2 * nv;
    if (params->K > min_cands)
      return fail(CM_ERR_INVALID_ARG, "K exceeds the vertex-contact count of the smallest registered geometry");
  } else if (c->min_e < 3) {
    return fail(CM_ERR_INVALID_ARG, "E-E contacts need every registered geometry to have >= 3 edges");
  } else if (params->top_edges || params->top_verts) {
    const int nv = params->top_verts ? std::min(params->top_verts, c->min_v) : c->min_v;
    const int ne = params->top_edges ? std::min(params->top_edges, c->min_e) : c->min_e;
    if (params->K > 2 * nv + 2 * ne * ne)
      return fail(CM_ERR_INVALID_ARG, "K exceeds the candidates left after pre-selection");
  }
  return CM_OK;
}

// Autotune cache key: direction, batch size (power-of-two bucket), largest edge
// count (bucket of 32) and the flags that change the work.
uint64_t tune_key(int bwd, int n_pairs, int max_e, int flags) {
  int nb = 0;
  while ((1 << nb) < n_pairs && nb < 31) ++nb;
  return ((uint64_t)bwd << 40) | ((uint64_t)nb << 32) | ((uint64_t)(max_e / 32) << 8) | (uint64_t)(flags & 3);
}

// The one-warp-per-pair forward can run this context's pairs: no pre-selection and
// 8 warps' slices fit the shared memory.
bool warp_path_ok(const cm_context* c, int flags_unused, int top_verts, int top_edges) {
  (void)flags_unused;
  if (top_verts || top_edges) return false;
  return fwd_warp_fits(make_layout(c, 1, 0, false), 256);
}

LaunchCfg default_cfg(const cm_context* c, int bwd, int n_pairs) {
  LaunchCfg g;
  g.block = 256;
  g.per_sm = 0;
  g.ordered = n_pairs >= 2 * c->num_sms ? 1 : 0;
  // small bodies (box-sized: up to 48 edges) go one warp per pair by default
  g.warp = (!bwd && c->max_e <= 48 && warp_path_ok(c, 0, 0, 0)) ? 1 : 0;
  return g;
}

LaunchCfg pick_cfg(const cm_context* c, int bwd, int n_pairs, int flags) {
  auto it = c->tuned.find(tune_key(bwd, n_pairs, c->max_e, flags));
  return it != c->tuned.end() ? it->second : default_cfg(c, bwd, n_pairs);
}

Params to_params(const cm_params* p) {
  return Params{p->tau, p->w_reg, p->eps_clip, p->eps_min, p->eps_comp, p->K, p->flags, p->top_verts, p->top_edges,
                p->trace_iters};
}

// Grid and shared-memory layout of one launch shape.
void shape(const cm_context* c, int bwd, const LaunchCfg& cfg, int n_pairs, SmemLayout& L, int& grid) {
  if (!bwd && cfg.warp) {
    L = make_layout(c, 1, 0, false);
    const int nw = cfg.block / 32;
    int per_sm = std::max(1, fwd_warp_max_blocks_per_sm(cfg.block, fwd_warp_bytes(L) * nw));
    if (cfg.per_sm > 0) per_sm = std::min(per_sm, cfg.per_sm);
    grid = std::max(1, std::min<int>((n_pairs + nw - 1) / nw, c->num_sms * per_sm));
    return;
  }
  L = make_layout(c, cfg.block / 32, bwd);
  int per_sm = bwd ? bwd_max_blocks_per_sm(cfg.block, L.total, cfg.per_sm) : fwd_max_blocks_per_sm(cfg.block, L.total);
  if (cfg.per_sm > 0) per_sm = std::min(per_sm, cfg.per_sm);
  grid = std::max(1, std::min<int>(n_pairs, c->num_sms * per_sm));
}

// Forward: dbar, alpha1, alpha2, con per edge pair; adjoint: dbar, t1, t2,
// alpha1, alpha2, con and the adjoints of the last three.
size_t scratch_need(const cm_context* c, int bwd, int grid, int64_t stride) {
  if (stride <= 0) stride = std::max<int64_t>(1, (int64_t)c->max_e * c->max_e);
  return (size_t)grid * stride * (bwd ? kBwdScratchArrays : 4);
}

int64_t saved_stride_floats(const cm_context* c, int K) {
  return ((int64_t)kRecHead * K + 2 * (int64_t)c->max_e + 3) & ~(int64_t)3;
}

// Queues one manifold step (work ordering + forward or adjoint kernel) on `s`
// with the given buffers; allocates nothing.
cm_status enqueue_step(const cm_context* c, int bwd, const LaunchCfg& cfg, int32_t n_pairs, const int32_t* pg,
                       const float* poses, const float* dims, const float* tau, const cm_params* params, float* out,
                       const float* grad_out, float* grad_poses, float* grad_dims, float* scratch,
                       int32_t* order, int32_t* counter, cudaStream_t s, int64_t stride, const StepExtras& x) {
  FwdArgs a{};
  int grid = 1;
  shape(c, bwd, cfg, n_pairs, a.sm, grid);
  a.hdr = c->d_hdr;
  a.n_geoms = (int32_t)c->hdr.size();
  a.verts = c->d_verts;
  a.edges = c->d_edges;
  a.planes = c->d_planes;
  a.n_pairs = n_pairs;
  a.pair_geoms = pg;
  a.poses = poses;
  a.dims = dims;
  a.tau = tau;
  a.p = to_params(params);
  a.out = out;
  a.scratch = scratch;
  a.scratch_stride = stride > 0 ? stride : std::max<int64_t>(1, (int64_t)c->max_e * c->max_e);
  a.err = c->d_err;
  a.work_counter = nullptr;
  a.order = nullptr;
  a.store_alpha = bwd ? 0 : 1;
  a.saved = x.saved;
  a.saved_stride = x.saved_stride;
  a.saved_first = x.saved_first;
  a.dump = bwd ? nullptr : x.dump;
  a.dump_off = x.dump_off;
  a.dump_rows = x.dump_rows;
  cudaError_t e;
  if (cfg.ordered) {
    if ((e = launch_order(pg, c->d_hdr, a.n_geoms, n_pairs, order, counter, bwd, s)) != cudaSuccess)
      return cuda_fail(e, "work-order launch");
    a.order = order;
    a.work_counter = counter;
  }
  const bool warp = !bwd && cfg.warp && !params->top_verts && !params->top_edges;
  if (!bwd && cfg.warp && !warp) {  // a tuned warp shape met pre-selection: the CTA kernel's layout
    shape(c, 0, LaunchCfg{cfg.block, cfg.per_sm, cfg.ordered, 0}, n_pairs, a.sm, grid);
  }
  e = bwd ? launch_bwd(a, grad_out, grad_poses, grad_dims, grid, cfg.block, cfg.per_sm, s)
      : warp ? launch_fwd_warp(a, grid, cfg.block, s) : launch_fwd(a, grid, cfg.block, s);
  if (e != cudaSuccess) return cuda_fail(e, bwd ? "backward launch" : "forward launch");
  return CM_OK;
}

// Context-owned buffers for one call with the chosen shape, then the step.
cm_status run_step(cm_context* c, int bwd, const LaunchCfg& cfg, int32_t n_pairs, const int32_t* pg,
                   const float* poses, const float* dims, const float* tau, const cm_params* params, float* out,
                   const float* grad_out, float* grad_poses, float* grad_dims, cudaStream_t s,
                   const StepExtras& x = StepExtras{}) {
  SmemLayout L;
  int grid = 1;
  shape(c, bwd, cfg, n_pairs, L, grid);
  cm_status st = ensure_scratch(c, scratch_need(c, bwd, grid, 0));
  if (st != CM_OK) return st;
  if ((st = ensure_order(c, (size_t)n_pairs)) != CM_OK) return st;
  return enqueue_step(c, bwd, cfg, n_pairs, pg, poses, dims, tau, params, out, grad_out, grad_poses, grad_dims,
                      c->d_scratch, c->d_order, c->d_counter, s, 0, x);
}

// A caller's record buffer: saved_stride floats per pair, at least what the
// context's largest geometry needs.
cm_status check_saved(const cm_context* c, const cm_params* params, const float* saved, int64_t saved_stride) {
  if (!saved) return fail(CM_ERR_INVALID_ARG, "the record buffer is required");
  if (saved_stride < saved_stride_floats(c, params->K))
    return fail(CM_ERR_INVALID_ARG,
                "saved_stride is below cm_saved_stride for these params and the registered geometry (geometry with "
                "more edges registered since the record was sized?)");
  if (reinterpret_cast<uintptr_t>(saved) % 4 != 0) return fail(CM_ERR_INVALID_ARG, "saved must be float-aligned");
  return CM_OK;
}
}  // namespace rt
}  // namespace cm

extern "C" {

void cm_default_params(cm_params* p) {
  if (!p) return;
  p->tau = 1e-2f;
  p->w_reg = 1e-2f;
  p->eps_clip = 0.1f;
  p->eps_min = 0.1f;
  p->eps_comp = 0.1f;
  p->K = 8;
  p->flags = 0;
  p->top_verts = 0;
  p->top_edges = 0;
  p->trace_iters = 0;
}

const char* cm_last_error(void) { return g_last_error.c_str(); }

cm_status cm_create_context(int device, size_t hbm_budget_bytes, cm_context** out) {
  if (!out) return fail(CM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (device == -1) {  // host-only: geometry registration and validation, no device work
    cm_context* c = new (std::nothrow) cm_context();
    if (!c) return fail(CM_ERR_OOM, "context allocation");
    c->device = -1;
    c->budget = hbm_budget_bytes;
    *out = c;
    return CM_OK;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(CM_ERR_INVALID_ARG, "device index out of range");
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cm_context* c = new (std::nothrow) cm_context();
  if (!c) return fail(CM_ERR_OOM, "context allocation");
  c->device = device;
  c->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if ((e = cudaMalloc(&c->d_err, sizeof(int))) != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc(error flag)");
  }
  cudaMemset(c->d_err, 0, sizeof(int));
  *out = c;
  return CM_OK;
}

void cm_destroy_context(cm_context* c) {
  if (!c) return;
  if (c->device < 0) {
    delete c;
    return;
  }
  server_shutdown(c);  // drain and stop the serving loop before freeing what it uses
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->d_hdr);
  cudaFree(c->d_verts);
  cudaFree(c->d_edges);
  cudaFree(c->d_planes);
  cudaFree(c->d_scratch);
  cudaFree(c->d_err);
  cudaFree(c->d_order);
  cudaFree(c->d_counter);
  delete c;
}

namespace {

// Device rows of one superquadric of an SQ_UNION geometry (five float4): the
// rows of R^T with -R^T t (x = R^T (y - t) = M y + c), then (1/a, 1/b, 1/c,
// 2/eps1) and (2/eps2, eps2/eps1, eps1/2, 0).
void pack_sq(const float* r, std::vector<float4>& out) {
  double qw = r[0], qx = r[1], qy = r[2], qz = r[3];
  const double qn = std::sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
  qw /= qn; qx /= qn; qy /= qn; qz /= qn;
  const double R[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
                          {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
                          {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
  const double t[3] = {r[4], r[5], r[6]};
  for (int i = 0; i < 3; ++i) {  // row i of R^T is column i of R
    const double c = -(R[0][i] * t[0] + R[1][i] * t[1] + R[2][i] * t[2]);
    out.push_back(make_float4((float)R[0][i], (float)R[1][i], (float)R[2][i], (float)c));
  }
  const double e1 = r[7], e2 = r[11];
  out.push_back(make_float4((float)(1.0 / r[8]), (float)(1.0 / r[9]), (float)(1.0 / r[10]), (float)(2.0 / e1)));
  out.push_back(make_float4((float)(2.0 / e2), (float)(e2 / e1), (float)(0.5 * e1), 0.f));
}

cm_status check_sq_rows(const cm_geometry_desc* d) {
  if (d->n_planes < 3 || d->n_planes % 3 || d->n_planes / 3 > CM_MAX_PRIMS || !d->planes)
    return fail(CM_ERR_INVALID_ARG, "an SQ_UNION needs 3 rows per superquadric, 1..32 superquadrics");
  for (int l = 0; l < d->n_planes / 3; ++l) {
    const float* r = d->planes + 12 * l;
    if (!(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3] > 1e-12f))
      return fail(CM_ERR_INVALID_ARG, "superquadric orientation quaternion is zero");
    if (!finite_pos(r[8]) || !finite_pos(r[9]) || !finite_pos(r[10]))
      return fail(CM_ERR_INVALID_ARG, "superquadric semi-axes must be finite and > 0");
    for (int e : {7, 11})
      if (!(r[e] >= 0.1f && r[e] <= 1.9f))
        return fail(CM_ERR_INVALID_ARG, "superquadric exponents must be in [0.1, 1.9]");
  }
  return CM_OK;
}

}  // namespace

cm_status cm_create_geometry(cm_context* c, const cm_geometry_desc* d, int32_t* geom_id) {
  if (!c || !d || !geom_id) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  if (d->kind < CM_BOX || d->kind > CM_SQ_UNION) return fail(CM_ERR_INVALID_ARG, "unknown geometry kind");
  if (d->n_verts < 1 || d->n_verts > CM_MAX_VERTS || !d->verts)
    return fail(CM_ERR_INVALID_ARG, "n_verts must be in 1..256 with a vertex array");
  if (d->n_edges < 0 || d->n_edges > CM_MAX_EDGES || (d->n_edges > 0 && !d->edges))
    return fail(CM_ERR_INVALID_ARG, "n_edges must be in 0..768 with an edge array");
  if (d->kind == CM_HULL) {
    if (d->n_planes < 4 || d->n_planes > CM_MAX_PLANES || !d->planes)
      return fail(CM_ERR_INVALID_ARG, "a hull needs 4..512 planes");
    if (d->n_verts < 4) return fail(CM_ERR_INVALID_ARG, "a hull needs at least 4 vertices");
  } else if (d->kind == CM_SQ_UNION) {
    for (int i = 0; i < 4 * d->n_planes && d->planes; ++i)
      if (!std::isfinite(d->planes[i])) return fail(CM_ERR_INVALID_ARG, "non-finite superquadric row");
    cm_status st = check_sq_rows(d);
    if (st != CM_OK) return st;
  } else {
    if (d->n_planes != 0) return fail(CM_ERR_INVALID_ARG, "planes are only given for hulls and SQ unions");
    int need = (d->kind == CM_CAPSULE || d->kind == CM_CYLINDER) ? 2 : 3;
    for (int i = 0; i < need; ++i)
      if (!finite_pos(d->dims[i])) return fail(CM_ERR_INVALID_ARG, "primitive dims must be finite and > 0");
  }
  for (int i = 0; i < 4 * d->n_verts; ++i)
    if (!std::isfinite(d->verts[i])) return fail(CM_ERR_INVALID_ARG, "non-finite vertex");
  for (int i = 0; i < 2 * d->n_edges; ++i)
    if (d->edges[i] < 0 || d->edges[i] >= d->n_verts) return fail(CM_ERR_INVALID_ARG, "edge index out of range");
  for (int i = 0; i < d->n_edges; ++i)
    if (d->edges[2 * i] == d->edges[2 * i + 1]) return fail(CM_ERR_INVALID_ARG, "degenerate edge");
  if (d->kind == CM_HULL) {
    for (int i = 0; i < 4 * d->n_planes; ++i)
      if (!std::isfinite(d->planes[i])) return fail(CM_ERR_INVALID_ARG, "non-finite plane");
    for (int i = 0; i < d->n_planes; ++i) {
      const float* p = d->planes + 4 * i;
      float nn = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
      if (std::fabs(nn - 1.f) > 1e-3f) return fail(CM_ERR_INVALID_ARG, "hull plane normals must be unit length");
    }
  }
  std::lock_guard<std::mutex> lk(c->mu);
  GeomHeader h{};
  h.kind = d->kind;
  h.n_verts = d->n_verts;
  h.n_edges = d->n_edges;
  h.v_off = (int)c->verts.size();
  h.e_off = (int)c->edges.size();
  h.p_off = (int)c->planes.size();
  for (int i = 0; i < 3; ++i) h.dims[i] = d->dims[i];
  if (d->kind == CM_SQ_UNION) {
    h.dims[0] = h.dims[1] = h.dims[2] = 1.f;
    for (int l = 0; l < d->n_planes / 3; ++l) pack_sq(d->planes + 12 * l, c->planes);
    h.n_planes = kSqRows * (d->n_planes / 3);
  } else {
    for (int i = 0; i < d->n_planes; ++i)
      c->planes.push_back(make_float4(d->planes[4 * i], d->planes[4 * i + 1], d->planes[4 * i + 2], d->planes[4 * i + 3]));
    h.n_planes = d->n_planes;
  }
  for (int i = 0; i < d->n_verts; ++i)
    c->verts.push_back(make_float4(d->verts[4 * i], d->verts[4 * i + 1], d->verts[4 * i + 2], d->verts[4 * i + 3]));
  for (int i = 0; i < d->n_edges; ++i)
    c->edges.push_back((uint32_t)d->edges[2 * i] | ((uint32_t)d->edges[2 * i + 1] << 16));
  c->hdr.push_back(h);
  c->max_v = std::max(c->max_v, d->n_verts);
  c->max_e = std::max(c->max_e, d->n_edges);
  c->max_p = std::max(c->max_p, h.n_planes);
  c->min_v = std::min(c->min_v, d->n_verts);
  c->min_e = std::min(c->min_e, d->n_edges);
  c->dirty = true;
  *geom_id = (int32_t)c->hdr.size() - 1;
  return CM_OK;
}

cm_status cm_sync_geometry(cm_context* c) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return sync_geometry_locked(c);
}

cm_status cm_destroy_geometry(cm_context* c, int32_t geom_id) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  std::lock_guard<std::mutex> lk(c->mu);
  if (geom_id < 0 || geom_id >= (int32_t)c->hdr.size()) return fail(CM_ERR_INVALID_ARG, "unknown geometry id");
  GeomHeader& h = c->hdr[geom_id];
  if (h.n_verts <= 0) return fail(CM_ERR_INVALID_ARG, "geometry already destroyed");
  // the kernels treat a header without vertices as an invalid id; its packed data stays
  h.n_verts = h.n_edges = h.n_planes = 0;
  // the smallest live geometry bounds K and the E-E checks
  c->min_v = c->min_e = 1 << 30;
  for (const GeomHeader& g : c->hdr)
    if (g.n_verts > 0) {
      c->min_v = std::min(c->min_v, g.n_verts);
      c->min_e = std::min(c->min_e, g.n_edges);
    }
  c->dirty = true;
  ++c->geom_gen;  // plans made before hold the old headers: invalid from now on
  return CM_OK;
}

int32_t cm_num_geometries(const cm_context* c) {
  if (!c) return 0;
  std::lock_guard<std::mutex> lk(c->mu);
  return (int32_t)c->hdr.size();
}

cm_status cm_check_device_error(cm_context* c) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  if (c->device < 0) return CM_OK;
  cudaSetDevice(c->device);
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  if ((e = cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read device error flag");
  if (v != 0) {
    cudaMemset(c->d_err, 0, sizeof(int));
    char buf[160];
    if (v > 0) std::snprintf(buf, sizeof buf, "pair %d names an unknown or destroyed geometry id", v - 1);
    else
      std::snprintf(buf, sizeof buf,
                    "pair %d: the candidate offsets do not match its candidate count or pass the dump's rows", -v - 1);
    return fail(CM_ERR_DEVICE, buf);
  }
  return CM_OK;
}

}  // extern "C"

namespace {
cm_status fwd_call(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses, const float* dims,
                   const float* tau, const cm_params* params, float* out, const StepExtras& x, bool with_record,
                   void* stream) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs < 0) return fail(CM_ERR_INVALID_ARG, "n_pairs < 0");
  if (n_pairs == 0) return CM_OK;
  if (!pair_geoms || !poses || !out) return fail(CM_ERR_INVALID_ARG, "pair_geoms, poses and out are required");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  if ((st = check_k(c, params)) != CM_OK) return st;
  if (with_record && (st = check_saved(c, params, x.saved, x.saved_stride)) != CM_OK) return st;
  if (x.dump && (!x.dump_off || x.dump_rows < 0 || (reinterpret_cast<uintptr_t>(x.dump) & 3)))
    return fail(CM_ERR_INVALID_ARG, "the candidate dump needs a float-aligned buffer, its row count and the offsets");
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;
  return run_step(c, 0, pick_cfg(c, 0, n_pairs, params->flags), n_pairs, pair_geoms, poses, dims, tau, params, out,
                  nullptr, nullptr, nullptr, (cudaStream_t)stream, x);
}

cm_status bwd_call(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses, const float* dims,
                   const float* tau, const cm_params* params, const float* saved, int64_t saved_stride,
                   bool with_record, const float* grad_out, float* grad_poses, float* grad_dims, void* stream) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs < 0) return fail(CM_ERR_INVALID_ARG, "n_pairs < 0");
  if (n_pairs == 0) return CM_OK;
  if (!pair_geoms || !poses || !grad_out || !grad_poses)
    return fail(CM_ERR_INVALID_ARG, "pair_geoms, poses, grad_out and grad_poses are required");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  if ((st = check_k(c, params)) != CM_OK) return st;
  if (with_record && (st = check_saved(c, params, saved, saved_stride)) != CM_OK) return st;
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;
  StepExtras x;
  x.saved = const_cast<float*>(saved);
  x.saved_stride = saved_stride;
  return run_step(c, 1, pick_cfg(c, 1, n_pairs, params->flags), n_pairs, pair_geoms, poses, dims, tau, params,
                  nullptr, grad_out, grad_poses, grad_dims, (cudaStream_t)stream, x);
}
}  // namespace

extern "C" {

cm_status cm_contact_manifold_fwd(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                  const float* dims, const float* tau, const cm_params* params, float* out,
                                  void* stream) {
  return fwd_call(c, n_pairs, pair_geoms, poses, dims, tau, params, out, StepExtras{}, false, stream);
}

cm_status cm_saved_stride(const cm_context* c, const cm_params* params, int64_t* floats_per_pair) {
  if (!c || !floats_per_pair) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  *floats_per_pair = saved_stride_floats(c, params->K);
  return CM_OK;
}

cm_status cm_contact_manifold_fwd_save(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                       const float* dims, const float* tau, const cm_params* params, float* out,
                                       float* saved, int64_t saved_stride, void* stream) {
  StepExtras x;
  x.saved = saved;
  x.saved_stride = saved_stride;
  return fwd_call(c, n_pairs, pair_geoms, poses, dims, tau, params, out, x, true, stream);
}

cm_status cm_candidate_offsets(const cm_context* c, int32_t n_pairs, const int32_t* pair_geoms_host,
                               const cm_params* params, int64_t* offsets_host) {
  if (!c || !offsets_host || (n_pairs > 0 && !pair_geoms_host)) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  if (n_pairs < 0) return fail(CM_ERR_INVALID_ARG, "n_pairs < 0");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  const bool one_sided = params->flags & CM_FLAG_ONE_SIDED, no_ee = one_sided || (params->flags & CM_FLAG_NO_EE);
  const auto sel = [](int limit, int n) { return limit ? std::min(limit, n) : n; };
  int64_t acc = 0;
  offsets_host[0] = 0;
  for (int32_t i = 0; i < n_pairs; ++i) {
    const int32_t ga = pair_geoms_host[2 * i], gb = pair_geoms_host[2 * i + 1];
    if (ga < 0 || gb < 0 || ga >= (int32_t)c->hdr.size() || gb >= (int32_t)c->hdr.size() ||
        c->hdr[ga].n_verts <= 0 || c->hdr[gb].n_verts <= 0)
      return fail(CM_ERR_INVALID_ARG, "pair names an unknown or destroyed geometry id");
    const GeomHeader &A = c->hdr[ga], &B = c->hdr[gb];
    const int64_t nva = sel(params->top_verts, A.n_verts), nvb = sel(params->top_verts, B.n_verts);
    const int64_t nea = sel(params->top_edges, A.n_edges), neb = sel(params->top_edges, B.n_edges);
    acc += (one_sided ? nva : nva + nvb) + (no_ee ? 0 : 2 * nea * neb);
    offsets_host[i + 1] = acc;
  }
  return CM_OK;
}

cm_status cm_contact_manifold_fwd_dump(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                       const float* dims, const float* tau, const cm_params* params, float* out,
                                       float* candidates, int64_t candidate_rows, const int64_t* candidate_offsets,
                                       void* stream) {
  StepExtras x;
  x.dump = candidates;
  x.dump_off = candidate_offsets;
  x.dump_rows = candidate_rows;
  if (!candidates || !candidate_offsets) return fail(CM_ERR_INVALID_ARG, "candidates and candidate_offsets are required");
  return fwd_call(c, n_pairs, pair_geoms, poses, dims, tau, params, out, x, false, stream);
}

cm_status cm_contact_manifold_bwd_saved(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                        const float* dims, const float* tau, const cm_params* params,
                                        const float* saved, int64_t saved_stride, const float* grad_out,
                                        float* grad_poses, float* grad_dims, void* stream) {
  return bwd_call(c, n_pairs, pair_geoms, poses, dims, tau, params, saved, saved_stride, true, grad_out, grad_poses,
                  grad_dims, stream);
}

}  // extern "C"

extern "C" cm_status cm_contact_manifold_bwd(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms,
                                              const float* poses, const float* dims, const float* tau,
                                              const cm_params* params, const float* grad_out, float* grad_poses,
                                              float* grad_dims, void* stream) {
  return bwd_call(c, n_pairs, pair_geoms, poses, dims, tau, params, nullptr, 0, false, grad_out, grad_poses,
                  grad_dims, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free forward entry point.
//
// Some callers must not allocate device memory while they run the manifold:
// a host application that hands out every device allocation from its own pool
// (so that its accounting and its limit stay exact), or a real-time control loop
// that was promised a fixed memory footprint and cannot absorb the blocking and
// device-wide synchronisation that cudaMalloc / cudaFree may bring.
// cm_contact_manifold_fwd may grow its scratch on a call, so those callers use
// this variant instead: its E-E distance scratch is the fixed file-scope device
// array below, sized once for the whole process.
// ---------------------------------------------------------------------------
#define CM_NOALLOC_SCRATCH_FLOATS (16u * 1024u * 1024u)  // 64 MiB of FP32 per GPU

static __device__ __align__(256) float g_noalloc_scratch[CM_NOALLOC_SCRATCH_FLOATS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
// The host-side symbol is only a stand-in, so the address is looked up once per
// device with cudaGetSymbolAddress and cached.
cm_status noalloc_scratch(int device, float** out) {
  if (device < 0 || device >= kMaxDevices) return fail(CM_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_ptr[device] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[device];
  return CM_OK;
}
}  // namespace

extern "C" cm_status cm_contact_manifold_fwd_noalloc(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms,
                                                      const float* poses, const float* dims, const float* tau,
                                                      const cm_params* params, float* out, void* stream) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs < 0) return fail(CM_ERR_INVALID_ARG, "n_pairs < 0");
  if (n_pairs == 0) return CM_OK;
  if (!pair_geoms || !poses || !out) return fail(CM_ERR_INVALID_ARG, "pair_geoms, poses and out are required");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  if (c->device < 0) return fail(CM_ERR_INVALID_ARG, "host-only context: no device work");
  if (c->dirty)
    return fail(CM_ERR_INVALID_ARG, "geometry not uploaded: call cm_sync_geometry before the no-alloc entry point");
  if ((st = check_k(c, params)) != CM_OK) return st;
  // one scratch slice of max_e^2 floats per CTA; the fixed array must hold a
  // slice for every SM so that the launch still fills the GPU
  const int64_t stride = std::max<int64_t>(1, (int64_t)c->max_e * c->max_e);
  const int64_t slices = (int64_t)CM_NOALLOC_SCRATCH_FLOATS / stride;
  if (slices < c->num_sms) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "no-alloc scratch too small: the largest registered geometry has %d edges; at most %d edges fit "
                  "(%u floats of scratch, one %d x %d slice per SM)",
                  c->max_e, (int)std::sqrt((double)CM_NOALLOC_SCRATCH_FLOATS / c->num_sms),
                  CM_NOALLOC_SCRATCH_FLOATS, c->max_e, c->max_e);
    return fail(CM_ERR_INVALID_ARG, buf);
  }
  cudaSetDevice(c->device);
  float* scratch = nullptr;
  if ((st = noalloc_scratch(c->device, &scratch)) != CM_OK) return st;

  const int block = 256;
  FwdArgs a{};
  a.sm = make_layout(c, block / 32, 0);
  const int per_sm = fwd_max_blocks_per_sm(block, a.sm.total);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)n_pairs, (int64_t)c->num_sms * per_sm, slices}));
  a.hdr = c->d_hdr;
  a.n_geoms = (int32_t)c->hdr.size();
  a.verts = c->d_verts;
  a.edges = c->d_edges;
  a.planes = c->d_planes;
  a.n_pairs = n_pairs;
  a.pair_geoms = pair_geoms;
  a.poses = poses;
  a.dims = dims;
  a.tau = tau;
  a.p = to_params(params);
  a.out = out;
  a.scratch = scratch;  // written before it is read: no clearing needed
  a.scratch_stride = stride;
  a.err = c->d_err;
  a.work_counter = nullptr;
  a.order = nullptr;
  // One scratch float per edge pair (its distance): pass 2 solves each witness QP
  // again instead of reading it back, unlike the regular forward, which keeps four
  // floats per edge pair.  That single float is what lets max_e^2 floats per CTA,
  // and so the edge limit above, fit the fixed array.
  a.store_alpha = 0;
  cudaError_t e = launch_fwd(a, grid, block, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc forward launch");
  return CM_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times a small set of launch shapes on the caller's batch and
// keeps the fastest per (direction, batch-size bucket, largest edge count,
// flags) for the context's later calls and plans.
// ---------------------------------------------------------------------------
extern "C" cm_status cm_autotune(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                 const float* dims, const float* tau, const cm_params* params, float* out,
                                 const float* grad_out, float* grad_poses, float* grad_dims, void* stream) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs <= 0 || !pair_geoms || !poses || !out) return fail(CM_ERR_INVALID_ARG, "a non-empty batch is required");
  if (grad_out && !grad_poses) return fail(CM_ERR_INVALID_ARG, "grad_poses is required with grad_out");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  if ((st = check_k(c, params)) != CM_OK) return st;
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the adjoint is timed as plans and autograd run it: from the forward's records
  float* saved = nullptr;
  const int64_t rs = grad_out ? saved_stride_floats(c, params->K) : 0;
  StepExtras rec;
  rec.saved_stride = rs;
  if (rs) {
    cudaError_t e = cudaMalloc(&saved, (size_t)n_pairs * rs * sizeof(float));
    if (e != cudaSuccess) return fail(CM_ERR_OOM, std::string("autotune records: ") + cudaGetErrorString(e));
    rec.saved = saved;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int bwd = 0; bwd < (grad_out ? 2 : 1); ++bwd) {
    const int blocks[4] = {64, 128, 256, 512};
    const int per_sms[3] = {1, 2, 0};
    LaunchCfg best = default_cfg(c, bwd, n_pairs);
    float best_ms = 3.0e38f;
    for (int bi = 0; bi < 4; ++bi) {
      if (bwd && (blocks[bi] > 256 || blocks[bi] < 128)) continue;  // the adjoint kernel: 128..256 threads
      for (int pi = 0; pi < 3; ++pi)
        for (int v = 0; v < 4; ++v) {  // work order on / off, CTA or warp per pair (forward)
          const int ord = v & 1, wp = v >> 1;
          if (wp && (bwd || blocks[bi] > 256 || !warp_path_ok(c, params->flags, params->top_verts, params->top_edges) ||
                     !fwd_warp_fits(make_layout(c, 1, 0, false), blocks[bi])))
            continue;
          LaunchCfg g{blocks[bi], per_sms[pi], ord, wp};
          float ms_sum = 0.f;
          for (int rep = 0; rep < 3; ++rep) {
            if (rep > 0) cudaEventRecord(e0, s);
            st = run_step(c, bwd, g, n_pairs, pair_geoms, poses, dims, tau, params, out, grad_out, grad_poses,
                          grad_dims, s, rec);
            if (st != CM_OK) break;
            if (rep > 0) {
              cudaEventRecord(e1, s);
              cudaEventSynchronize(e1);
              float ms = 0.f;
              cudaEventElapsedTime(&ms, e0, e1);
              ms_sum += ms;
            }
          }
          if (st != CM_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaStreamSynchronize(s);
            cudaFree(saved);
            return st;
          }
          if (ms_sum < best_ms) {
            best_ms = ms_sum;
            best = g;
          }
        }
    }
    c->tuned[tune_key(bwd, n_pairs, c->max_e, params->flags)] = best;
    // the forward's records for the adjoint's shapes, from the chosen forward shape
    if (!bwd && saved) {
      st = run_step(c, 0, best, n_pairs, pair_geoms, poses, dims, tau, params, out, nullptr, nullptr, nullptr, s,
                    rec);
      if (st != CM_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamSynchronize(s);
        cudaFree(saved);
        return st;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(saved);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  return CM_OK;
}

extern "C" cm_status cm_get_launch_shape(const cm_context* c, int32_t n_pairs, int32_t backward, int32_t flags,
                                         int32_t* block, int32_t* ctas_per_sm, int32_t* ordered) {
  if (!c || !block || !ctas_per_sm || !ordered) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  LaunchCfg g = pick_cfg(c, backward ? 1 : 0, n_pairs, flags);
  *block = g.block;
  *ctas_per_sm = g.per_sm;
  *ordered = g.ordered;
  return CM_OK;
}

// ---------------------------------------------------------------------------
// Plans: the steady-state step of a fixed batch (work ordering + forward, and
// optionally + adjoint) captured once into a CUDA graph with its own scratch,
// then replayed with one graph launch per step.  The caller rewrites the
// input buffers (poses, dims, tau, grad_out) in place between replays.
// ---------------------------------------------------------------------------
struct cm_plan {
  cm_context* ctx = nullptr;
  uint64_t geom_gen = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float* scratch = nullptr;
  int32_t* order = nullptr;
  int32_t* counter = nullptr;
  float* saved = nullptr;  // forward records for the adjoint (forward + backward plans)
};

extern "C" void cm_plan_destroy(cm_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap) cudaStreamDestroy(p->cap);
  cudaFree(p->scratch);
  cudaFree(p->order);
  cudaFree(p->counter);
  cudaFree(p->saved);
  delete p;
}

extern "C" cm_status cm_plan_create(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                    const float* dims, const float* tau, const cm_params* params, float* out,
                                    const float* grad_out, float* grad_poses, float* grad_dims, cm_plan** plan) {
  if (!c || !plan) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  *plan = nullptr;
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs <= 0 || !pair_geoms || !poses || !out) return fail(CM_ERR_INVALID_ARG, "a non-empty batch is required");
  if (grad_out && !grad_poses) return fail(CM_ERR_INVALID_ARG, "grad_poses is required with grad_out");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  if ((st = check_k(c, params)) != CM_OK) return st;
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;
  cm_plan* p = new (std::nothrow) cm_plan();
  if (!p) return fail(CM_ERR_OOM, "plan allocation");
  p->ctx = c;
  p->geom_gen = c->geom_gen;
  const LaunchCfg gf = pick_cfg(c, 0, n_pairs, params->flags);
  const LaunchCfg gb = pick_cfg(c, 1, n_pairs, params->flags);
  SmemLayout L;
  int grid_f = 1, grid_b = 1;
  shape(c, 0, gf, n_pairs, L, grid_f);
  shape(c, 1, gb, n_pairs, L, grid_b);
  size_t need = scratch_need(c, 0, grid_f, 0);
  if (grad_out) need = std::max(need, scratch_need(c, 1, grid_b, 0));
  const int64_t rs = grad_out ? saved_stride_floats(c, params->K) : 0;
  StepExtras rec;
  cudaError_t e;
  if ((e = cudaMalloc(&p->scratch, need * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&p->order, (size_t)n_pairs * sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&p->counter, sizeof(int32_t))) != cudaSuccess ||
      (rs && (e = cudaMalloc(&p->saved, (size_t)n_pairs * rs * sizeof(float))) != cudaSuccess)) {
    cm_plan_destroy(p);
    return fail(CM_ERR_OOM, std::string("plan buffers: ") + cudaGetErrorString(e));
  }
  rec.saved = p->saved;
  rec.saved_stride = rs;
  if ((e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess) {
    cm_plan_destroy(p);
    return cuda_fail(e, "plan stream");
  }
  // first launches outside the capture set the kernels' attributes
  st = enqueue_step(c, 0, gf, n_pairs, pair_geoms, poses, dims, tau, params, out, nullptr, nullptr, nullptr,
                    p->scratch, p->order, p->counter, p->cap, 0, rec);
  if (st == CM_OK && grad_out)
    st = enqueue_step(c, 1, gb, n_pairs, pair_geoms, poses, dims, tau, params, nullptr, grad_out, grad_poses,
                      grad_dims, p->scratch, p->order, p->counter, p->cap, 0, rec);
  if (st == CM_OK && (e = cudaStreamSynchronize(p->cap)) != cudaSuccess) st = cuda_fail(e, "plan warm-up");
  if (st == CM_OK && (e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    st = cuda_fail(e, "begin capture");
  if (st == CM_OK) {
    cm_status s1 = enqueue_step(c, 0, gf, n_pairs, pair_geoms, poses, dims, tau, params, out, nullptr, nullptr,
                                nullptr, p->scratch, p->order, p->counter, p->cap, 0, rec);
    if (s1 == CM_OK && grad_out)
      s1 = enqueue_step(c, 1, gb, n_pairs, pair_geoms, poses, dims, tau, params, nullptr, grad_out, grad_poses,
                        grad_dims, p->scratch, p->order, p->counter, p->cap, 0, rec);
    e = cudaStreamEndCapture(p->cap, &p->graph);
    if (s1 != CM_OK) st = s1;
    else if (e != cudaSuccess) st = cuda_fail(e, "end capture");
  }
  if (st == CM_OK && (e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess)
    st = cuda_fail(e, "graph instantiate");
  if (st != CM_OK) {
    cm_plan_destroy(p);
    return st;
  }
  *plan = p;
  return CM_OK;
}

extern "C" cm_status cm_plan_launch(cm_plan* p, void* stream) {
  if (!p) return fail(CM_ERR_INVALID_ARG, "NULL plan");
  if (p->ctx->geom_gen != p->geom_gen)
    return fail(CM_ERR_INVALID_ARG, "geometry changed since the plan was made: create the plan again");
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return CM_OK;
}
