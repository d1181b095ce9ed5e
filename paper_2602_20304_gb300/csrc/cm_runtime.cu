// cm_runtime.cu -- host side of the C ABI declared in include/contact_manifold.h:
// context, packed geometry store, argument validation, scratch management and
// kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "contact_manifold.h"
#include "cm_internal.h"

using namespace cm;

namespace {
thread_local std::string g_last_error;

cm_status fail(cm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
cm_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
int align16(int x) { return (x + 15) & ~15; }
}  // namespace

struct cm_context {
  int device = 0;
  size_t budget = 0;
  int num_sms = 0;
  std::mutex mu;
  // host copy of the packed geometry store
  std::vector<GeomHeader> hdr;
  std::vector<float4> verts;
  std::vector<uint32_t> edges;
  std::vector<float4> planes;
  int max_v = 0, max_e = 0, max_p = 0, min_v = 1 << 30, min_e = 1 << 30;
  bool dirty = false;
  // device copy
  GeomHeader* d_hdr = nullptr;
  float4* d_verts = nullptr;
  uint32_t* d_edges = nullptr;
  float4* d_planes = nullptr;
  size_t cap_hdr = 0, cap_verts = 0, cap_edges = 0, cap_planes = 0;
  // scratch for the E-E distance matrix (per CTA slice) and the error flag
  float* d_scratch = nullptr;
  size_t scratch_floats = 0;
  int* d_err = nullptr;
};

namespace {

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
  if (!c->dirty) return CM_OK;
  cudaError_t e;
  if ((e = grow_upload(c->d_hdr, c->cap_hdr, c->hdr)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  if ((e = grow_upload(c->d_verts, c->cap_verts, c->verts)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  if ((e = grow_upload(c->d_edges, c->cap_edges, c->edges)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  if ((e = grow_upload(c->d_planes, c->cap_planes, c->planes)) != cudaSuccess) return cuda_fail(e, "geometry upload");
  c->dirty = false;
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
  if (p->flags & ~3) return fail(CM_ERR_INVALID_ARG, "unknown flag bits");
  return CM_OK;
}

SmemLayout make_layout(const cm_context* c, int nwarps) {
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

}  // namespace

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
}

const char* cm_last_error(void) { return g_last_error.c_str(); }

cm_status cm_create_context(int device, size_t hbm_budget_bytes, cm_context** out) {
  if (!out) return fail(CM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
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
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->d_hdr);
  cudaFree(c->d_verts);
  cudaFree(c->d_edges);
  cudaFree(c->d_planes);
  cudaFree(c->d_scratch);
  cudaFree(c->d_err);
  delete c;
}

cm_status cm_create_geometry(cm_context* c, const cm_geometry_desc* d, int32_t* geom_id) {
  if (!c || !d || !geom_id) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  if (d->kind < CM_BOX || d->kind > CM_HULL) return fail(CM_ERR_INVALID_ARG, "unknown geometry kind");
  if (d->n_verts < 1 || d->n_verts > CM_MAX_VERTS || !d->verts)
    return fail(CM_ERR_INVALID_ARG, "n_verts must be in 1..256 with a vertex array");
  if (d->n_edges < 0 || d->n_edges > CM_MAX_EDGES || (d->n_edges > 0 && !d->edges))
    return fail(CM_ERR_INVALID_ARG, "n_edges must be in 0..768 with an edge array");
  if (d->kind == CM_HULL) {
    if (d->n_planes < 4 || d->n_planes > CM_MAX_PLANES || !d->planes)
      return fail(CM_ERR_INVALID_ARG, "a hull needs 4..512 planes");
    if (d->n_verts < 4) return fail(CM_ERR_INVALID_ARG, "a hull needs at least 4 vertices");
  } else {
    if (d->n_planes != 0) return fail(CM_ERR_INVALID_ARG, "planes are only given for hulls");
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
  for (int i = 0; i < 4 * d->n_planes; ++i)
    if (!std::isfinite(d->planes[i])) return fail(CM_ERR_INVALID_ARG, "non-finite plane");
  for (int i = 0; i < d->n_planes; ++i) {
    const float* p = d->planes + 4 * i;
    float nn = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    if (std::fabs(nn - 1.f) > 1e-3f) return fail(CM_ERR_INVALID_ARG, "hull plane normals must be unit length");
  }
  std::lock_guard<std::mutex> lk(c->mu);
  GeomHeader h{};
  h.kind = d->kind;
  h.n_verts = d->n_verts;
  h.n_edges = d->n_edges;
  h.n_planes = d->n_planes;
  h.v_off = (int)c->verts.size();
  h.e_off = (int)c->edges.size();
  h.p_off = (int)c->planes.size();
  for (int i = 0; i < 3; ++i) h.dims[i] = d->dims[i];
  for (int i = 0; i < d->n_verts; ++i)
    c->verts.push_back(make_float4(d->verts[4 * i], d->verts[4 * i + 1], d->verts[4 * i + 2], d->verts[4 * i + 3]));
  for (int i = 0; i < d->n_edges; ++i)
    c->edges.push_back((uint32_t)d->edges[2 * i] | ((uint32_t)d->edges[2 * i + 1] << 16));
  for (int i = 0; i < d->n_planes; ++i)
    c->planes.push_back(make_float4(d->planes[4 * i], d->planes[4 * i + 1], d->planes[4 * i + 2], d->planes[4 * i + 3]));
  c->hdr.push_back(h);
  c->max_v = std::max(c->max_v, d->n_verts);
  c->max_e = std::max(c->max_e, d->n_edges);
  c->max_p = std::max(c->max_p, d->n_planes);
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

int32_t cm_num_geometries(const cm_context* c) { return c ? (int32_t)c->hdr.size() : 0; }

cm_status cm_check_device_error(cm_context* c) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cudaSetDevice(c->device);
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  if ((e = cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read device error flag");
  if (v != 0) {
    cudaMemset(c->d_err, 0, sizeof(int));
    char buf[128];
    std::snprintf(buf, sizeof buf, "pair %d names an unknown geometry id", v - 1);
    return fail(CM_ERR_DEVICE, buf);
  }
  return CM_OK;
}

cm_status cm_contact_manifold_fwd(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms, const float* poses,
                                  const float* dims, const float* tau, const cm_params* params, float* out,
                                  void* stream) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs < 0) return fail(CM_ERR_INVALID_ARG, "n_pairs < 0");
  if (n_pairs == 0) return CM_OK;
  if (!pair_geoms || !poses || !out) return fail(CM_ERR_INVALID_ARG, "pair_geoms, poses and out are required");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  // every pair must offer at least K candidates: with E-E contacts any two
  // geometries of >= 3 edges give 2 * 3 * 3 = 18 > CM_MAX_K; without them the
  // vertex count of the smallest registered geometry bounds it
  if (params->flags & (CM_FLAG_NO_EE | CM_FLAG_ONE_SIDED)) {
    const int min_cands = (params->flags & CM_FLAG_ONE_SIDED) ? c->min_v : 2 * c->min_v;
    if (params->K > min_cands)
      return fail(CM_ERR_INVALID_ARG, "K exceeds the vertex-contact count of the smallest registered geometry");
  } else if (c->min_e < 3) {
    return fail(CM_ERR_INVALID_ARG, "E-E contacts need every registered geometry to have >= 3 edges");
  }
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;

  const int block = 256;
  FwdArgs a{};
  a.sm = make_layout(c, block / 32);
  const int per_sm = fwd_max_blocks_per_sm(block, a.sm.total);
  const int grid = std::max(1, std::min<int>(n_pairs, c->num_sms * per_sm));
  const int64_t stride = std::max<int64_t>(1, (int64_t)c->max_e * c->max_e);
  if ((st = ensure_scratch(c, (size_t)grid * stride)) != CM_OK) return st;

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
  a.p = Params{params->tau, params->w_reg, params->eps_clip, params->eps_min, params->eps_comp, params->K, params->flags};
  a.out = out;
  a.scratch = c->d_scratch;
  a.scratch_stride = stride;
  a.err = c->d_err;
  a.work_counter = nullptr;
  a.order = nullptr;
  cudaError_t e = launch_fwd(a, grid, block, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  return CM_OK;
}

}  // extern "C"

extern "C" cm_status cm_contact_manifold_bwd(cm_context* c, int32_t n_pairs, const int32_t* pair_geoms,
                                              const float* poses, const float* dims, const float* tau,
                                              const cm_params* params, const float* grad_out, float* grad_poses,
                                              float* grad_dims, void* stream) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (n_pairs < 0) return fail(CM_ERR_INVALID_ARG, "n_pairs < 0");
  if (n_pairs == 0) return CM_OK;
  if (!pair_geoms || !poses || !grad_out || !grad_poses)
    return fail(CM_ERR_INVALID_ARG, "pair_geoms, poses, grad_out and grad_poses are required");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "no geometry registered");
  if (params->flags & (CM_FLAG_NO_EE | CM_FLAG_ONE_SIDED)) {
    const int min_cands = (params->flags & CM_FLAG_ONE_SIDED) ? c->min_v : 2 * c->min_v;
    if (params->K > min_cands)
      return fail(CM_ERR_INVALID_ARG, "K exceeds the vertex-contact count of the smallest registered geometry");
  } else if (c->min_e < 3) {
    return fail(CM_ERR_INVALID_ARG, "E-E contacts need every registered geometry to have >= 3 edges");
  }
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;
  const int block = 256;
  FwdArgs a{};
  a.sm = make_layout(c, block / 32);
  const int per_sm = bwd_max_blocks_per_sm(block, a.sm.total);
  const int grid = std::max(1, std::min<int>(n_pairs, c->num_sms * per_sm));
  const int64_t stride = std::max<int64_t>(1, (int64_t)c->max_e * c->max_e);
  if ((st = ensure_scratch(c, (size_t)grid * stride * 3)) != CM_OK) return st;
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
  a.p = Params{params->tau, params->w_reg, params->eps_clip, params->eps_min, params->eps_comp, params->K, params->flags};
  a.out = nullptr;
  a.scratch = c->d_scratch;
  a.scratch_stride = stride;
  a.err = c->d_err;
  cudaError_t e = launch_bwd(a, grad_out, grad_poses, grad_dims, grid, block, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward launch");
  return CM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free forward entry point.
//
// Some callers must not allocate device memory while they run the manifold:
// a simulator stepping inside a CUDA stream capture (cudaMalloc is not allowed
// there), a real-time control loop that was promised a fixed memory footprint,
// or a host application that owns every device allocation through its own
// pool.  cm_contact_manifold_fwd may grow its scratch on a call, so those
// callers use this variant instead: its E-E distance scratch is the fixed
// file-scope device array below, sized once for the whole process.
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
  if (c->dirty)
    return fail(CM_ERR_INVALID_ARG, "geometry not uploaded: call cm_sync_geometry before the no-alloc entry point");
  if (params->flags & (CM_FLAG_NO_EE | CM_FLAG_ONE_SIDED)) {
    const int min_cands = (params->flags & CM_FLAG_ONE_SIDED) ? c->min_v : 2 * c->min_v;
    if (params->K > min_cands)
      return fail(CM_ERR_INVALID_ARG, "K exceeds the vertex-contact count of the smallest registered geometry");
  } else if (c->min_e < 3) {
    return fail(CM_ERR_INVALID_ARG, "E-E contacts need every registered geometry to have >= 3 edges");
  }
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
  a.sm = make_layout(c, block / 32);
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
  a.p = Params{params->tau, params->w_reg, params->eps_clip, params->eps_min, params->eps_comp, params->K, params->flags};
  a.out = out;
  a.scratch = scratch;  // written before it is read: no clearing needed
  a.scratch_stride = stride;
  a.err = c->d_err;
  a.work_counter = nullptr;
  a.order = nullptr;
  cudaError_t e = launch_fwd(a, grid, block, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc forward launch");
  return CM_OK;
}
