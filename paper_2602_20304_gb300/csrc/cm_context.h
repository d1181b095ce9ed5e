// cm_context.h -- the library context and the host helpers shared by the
// runtime (cm_runtime.cu) and the serving loop (cm_serve.cu).
#pragma once

#include <condition_variable>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "contact_manifold.h"
#include "cm_internal.h"

namespace cm {
struct Server;
}

struct cm_context {
  int device = 0;
  size_t budget = 0;
  int num_sms = 0;
  mutable std::mutex mu;  // also taken by the read-only calls
  // host copy of the packed geometry store
  std::vector<cm::GeomHeader> hdr;
  std::vector<float4> verts;
  std::vector<uint32_t> edges;
  std::vector<float4> planes;
  int max_v = 0, max_e = 0, max_p = 0, min_v = 1 << 30, min_e = 1 << 30;
  bool dirty = false;
  // device copy
  cm::GeomHeader* d_hdr = nullptr;
  float4* d_verts = nullptr;
  uint32_t* d_edges = nullptr;
  float4* d_planes = nullptr;
  size_t cap_hdr = 0, cap_verts = 0, cap_edges = 0, cap_planes = 0;
  // scratch for the E-E distance matrix (per CTA slice) and the error flag
  float* d_scratch = nullptr;
  size_t scratch_floats = 0;
  int* d_err = nullptr;
  // size-ordered work list of the last batch and its atomic counter
  int32_t* d_order = nullptr;
  size_t cap_order = 0;
  int32_t* d_counter = nullptr;
  uint64_t geom_gen = 0;                 // bumped by every geometry upload
  std::map<uint64_t, cm::LaunchCfg> tuned;  // autotuned launch shapes
  std::unique_ptr<cm::Server> server;    // serving loop (cm_server_start)
  cm_context();
  ~cm_context();
};

namespace cm {
namespace rt {
cm_status fail(cm_status s, const std::string& msg);
cm_status cuda_fail(cudaError_t e, const char* what);
cm_status sync_geometry_locked(cm_context* c);
cm_status check_params(const cm_params* p);
cm_status check_k(const cm_context* c, const cm_params* params);
LaunchCfg pick_cfg(const cm_context* c, int bwd, int n_pairs, int flags);
void shape(const cm_context* c, int bwd, const LaunchCfg& cfg, int n_pairs, SmemLayout& L, int& grid);
size_t scratch_need(const cm_context* c, int bwd, int grid, int64_t stride);  // stride <= 0: max_e^2
cm_status enqueue_step(const cm_context* c, int bwd, const LaunchCfg& cfg, int32_t n_pairs, const int32_t* pg,
                       const float* poses, const float* dims, const float* tau, const cm_params* params, float* out,
                       const float* grad_out, float* grad_poses, float* grad_dims, float* scratch,
                       int32_t* order, int32_t* counter, cudaStream_t s, int64_t stride,  // stride <= 0: max_e^2
                       const StepExtras& x = StepExtras{});  // forward records, candidate dump (optional)
// Floats per pair of the forward's record for the adjoint (see kRecHead).
int64_t saved_stride_floats(const cm_context* c, int K);
void server_shutdown(cm_context* c);  // cm_serve.cu
}  // namespace rt
}  // namespace cm
