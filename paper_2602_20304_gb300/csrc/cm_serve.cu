// cm_serve.cu -- serving loop: continuous batching of contact-manifold requests.
//
// Clients submit requests (a set of body pairs, forward or forward+backward)
// from any thread.  One scheduler thread per context
//   * admits queued requests in arrival order while their device memory fits
//     the context's HBM budget, the device's free memory and the batch's pair limit,
//   * packs each admitted group into one batch (forward-only requests first,
//     forward+backward requests as a contiguous tail), copies its inputs to the
//     device, runs work ordering + forward over the whole batch and ordering +
//     adjoint over the tail, and copies the results back, all on one of
//     several streams, so batches formed while others run overlap on the GPU,
//   * retires batches whose completion event has fired, frees their memory and
//     wakes the waiting clients.
// Geometry stays resident in the context; only per-request pair data moves.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>

#include "cm_context.h"

using namespace cm;
using namespace cm::rt;

namespace cm {

namespace {
using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  cm_request_desc d{};
  int64_t max_ee = 1;        // largest E_A x E_B among its pairs (scratch slice size)
  Clock::time_point t_submit, t_done;
  int state = 0;             // 0 queued, 1 running, 2 done, 3 failed
  cm_status status = CM_OK;
};

struct Batch {
  std::vector<Request*> reqs;
  int64_t max_ee = 1;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* mem = nullptr;       // one device block for every buffer of the batch
  size_t bytes = 0;
};

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Device bytes of one batch's block, exactly as Server::issue carves it: n pairs
// of which nb with the adjoint, `grid` scratch slices of max_ee edge pairs (the
// adjoint's kBwdScratchArrays floats each with an adjoint in the batch, else 4),
// the forward's records of the nb adjoint pairs (rec_floats each), the work list
// and its counter.
size_t batch_layout_bytes(size_t n, size_t nb, int K, size_t grid, int64_t max_ee, int64_t rec_floats) {
  const size_t nb1 = std::max<size_t>(nb, 1);
  return round256(8 * n) + round256(56 * n) + round256(24 * n) + round256(4 * n) + round256(32 * K * n) +
         round256(32 * K * nb1) + round256(56 * nb1) + round256(24 * nb1) +
         round256(grid * (size_t)max_ee * (nb ? kBwdScratchArrays : 4) * sizeof(float)) +
         round256(nb * (size_t)rec_floats * sizeof(float)) + round256(4 * n) + round256(4);
}
}  // namespace

struct Server {
  cm_context* ctx = nullptr;
  cm_params params{};
  int max_batch_pairs = 0;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_busy;
  cudaMemPool_t mempool = nullptr;  // this server's stream-ordered pool of batch blocks
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::unique_ptr<Batch>> running;
  uint64_t next_ticket = 1;
  size_t bytes_in_use = 0;
  int grid_max = 1;          // most CTAs any launch shape of a batch uses
  bool stop = false;
  std::thread thread;
  uint64_t pairs_done = 0, batches_done = 0;

  ~Server() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_work.notify_all();
    if (thread.joinable()) thread.join();
    for (auto& b : running) {
      cudaEventSynchronize(b->done);
      cudaEventDestroy(b->done);
      cudaFreeAsync(b->mem, b->stream);
    }
    for (cudaStream_t s : streams) cudaStreamSynchronize(s);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
    if (mempool) cudaMemPoolDestroy(mempool);  // returns the cached blocks to the driver
  }

  size_t budget() const { return ctx->budget ? ctx->budget : (size_t)1 << 62; }

  // Device block of a batch of `pairs` pairs (`bwd_pairs` with the adjoint) whose
  // largest E_A x E_B is max_ee (a launch never has more CTAs than pairs).
  size_t batch_bytes(int pairs, int bwd_pairs, int64_t max_ee) const {
    const size_t grid = (size_t)std::min(grid_max, std::max(pairs, 1));
    return batch_layout_bytes((size_t)std::max(pairs, 1), (size_t)bwd_pairs, params.K, grid, max_ee,
                              saved_stride_floats(ctx, params.K));
  }

  // Runs in the scheduler thread with `mu` held on entry and exit.
  void retire_finished(std::unique_lock<std::mutex>&) {
    for (size_t i = 0; i < running.size();) {
      Batch* b = running[i].get();
      cudaError_t q = cudaEventQuery(b->done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      const auto now = Clock::now();
      for (Request* r : b->reqs) {
        r->state = q == cudaSuccess ? 2 : 3;
        r->status = q == cudaSuccess ? CM_OK : CM_ERR_CUDA;
        r->t_done = now;
        pairs_done += (uint64_t)r->d.n_pairs;
      }
      ++batches_done;
      bytes_in_use -= b->bytes;
      for (size_t s = 0; s < streams.size(); ++s)
        if (streams[s] == b->stream) stream_busy[s] = 0;
      cudaEventDestroy(b->done);
      cudaFreeAsync(b->mem, b->stream);  // stream-ordered: no device-wide synchronisation
      running.erase(running.begin() + i);
      cv_done.notify_all();
    }
  }

  // Device memory a new batch block can take now: what the device has free plus
  // what the stream-ordered pool holds cached but unused, less a reserve for the
  // driver and the other users of this GPU.
  size_t free_hbm() const {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(mempool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(mempool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
      fr += (size_t)(reserved - used);
    return fr > kHbmReserve ? fr - kHbmReserve : 0;
  }
  static constexpr size_t kHbmReserve = (size_t)256 << 20;

  // Takes the longest admissible prefix of the queue; nullptr if nothing fits now.
  // A request is admitted while the batch fits both the context's budget (with
  // the batches already running) and the device's free memory.  A request that
  // cannot fit the free memory with nothing running fails with CM_ERR_ADMISSION
  // instead of waiting for memory that no batch of this server will release.
  std::unique_ptr<Batch> form_batch() {
    if (queue.empty()) return nullptr;
    int s = -1;
    for (size_t i = 0; i < streams.size(); ++i)
      if (!stream_busy[i]) {
        s = (int)i;
        break;
      }
    if (s < 0) return nullptr;
    const size_t avail = free_hbm();
    auto b = std::make_unique<Batch>();
    int pairs = 0, bwd_pairs = 0;
    int64_t mee = 1;
    size_t bytes = 0;
    while (!queue.empty()) {
      Request* r = queue.front();
      if (!b->reqs.empty() && pairs + r->d.n_pairs > max_batch_pairs) break;
      const int64_t m2 = std::max(mee, r->max_ee);
      const int nb2 = bwd_pairs + (r->d.with_backward ? r->d.n_pairs : 0);
      const size_t total = batch_bytes(pairs + r->d.n_pairs, nb2, m2);
      if (total > avail && b->reqs.empty() && running.empty()) {
        r->state = 3;
        r->status = CM_ERR_ADMISSION;
        r->t_done = Clock::now();
        queue.pop_front();
        cv_done.notify_all();
        continue;
      }
      if (bytes_in_use + total > budget() || total > avail) break;
      pairs += r->d.n_pairs;
      bwd_pairs = nb2;
      mee = m2;
      bytes = total;
      b->reqs.push_back(r);
      queue.pop_front();
    }
    if (b->reqs.empty()) return nullptr;
    b->stream = streams[s];
    stream_busy[s] = 1;
    b->bytes = bytes;
    b->max_ee = mee;
    bytes_in_use += bytes;
    return b;
  }

  // Issues a batch on its stream (called without `mu`).  Returns false on failure.
  cm_status issue(Batch* b) {
    // forward-only requests first, forward+backward ones as a contiguous tail
    std::stable_partition(b->reqs.begin(), b->reqs.end(), [](Request* r) { return !r->d.with_backward; });
    const int K = params.K;
    size_t n = 0, nb = 0;
    for (Request* r : b->reqs) {
      n += r->d.n_pairs;
      if (r->d.with_backward) nb += r->d.n_pairs;
    }
    cudaError_t e = cudaMallocFromPoolAsync(&b->mem, b->bytes, mempool, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch memory");
    char* p = static_cast<char*>(b->mem);
    auto take = [&](size_t bytes) {
      char* q = p;
      p += round256(bytes);
      return q;
    };
    int32_t* pg = (int32_t*)take(8 * n);
    float* poses = (float*)take(56 * n);
    float* dims = (float*)take(24 * n);
    float* tau = (float*)take(4 * n);
    float* out = (float*)take(32 * K * n);
    float* gout = (float*)take(32 * K * std::max<size_t>(nb, 1));
    float* gp = (float*)take(56 * std::max<size_t>(nb, 1));
    float* gd = (float*)take(24 * std::max<size_t>(nb, 1));
    const size_t grid = (size_t)std::min(grid_max, (int)std::max<size_t>(n, 1));
    float* scratch = (float*)take(grid * (size_t)b->max_ee * (nb ? kBwdScratchArrays : 4) * sizeof(float));
    const int64_t rs = saved_stride_floats(ctx, K);
    float* saved = (float*)take(nb * (size_t)rs * sizeof(float));
    int32_t* order = (int32_t*)take(4 * n);
    int32_t* counter = (int32_t*)take(4);
    if ((size_t)(p - static_cast<char*>(b->mem)) > b->bytes)  // the admission size and the carve disagree
      return fail(CM_ERR_INVALID_ARG, "internal: batch layout exceeds its block");
    cudaStream_t s = b->stream;
    // inputs
    size_t off = 0, offb = 0;
    for (Request* r : b->reqs) {
      const size_t m = (size_t)r->d.n_pairs;
      cudaMemcpyAsync(pg + 2 * off, r->d.pair_geoms, 8 * m, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(poses + 14 * off, r->d.poses, 56 * m, cudaMemcpyHostToDevice, s);
      if (r->d.dims) cudaMemcpyAsync(dims + 6 * off, r->d.dims, 24 * m, cudaMemcpyHostToDevice, s);
      if (r->d.tau) {
        cudaMemcpyAsync(tau + off, r->d.tau, 4 * m, cudaMemcpyHostToDevice, s);
      }
      if (r->d.with_backward) {
        cudaMemcpyAsync(gout + (size_t)8 * K * offb, r->d.grad_out, 32 * K * m, cudaMemcpyHostToDevice, s);
        offb += m;
      }
      off += m;
    }
    // per-request defaults for absent dims / tau are filled on the host side:
    // submit() rejects mixing, so either every request of the server gives them or none
    cm_status st;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      if ((st = sync_geometry_locked(ctx)) != CM_OK) return st;
      if (nb && saved_stride_floats(ctx, K) > rs)  // geometry with more edges registered since the block was sized
        return fail(CM_ERR_INVALID_ARG, "geometry changed while the batch was formed: its records no longer fit");
      const bool has_dims = b->reqs.front()->d.dims != nullptr, has_tau = b->reqs.front()->d.tau != nullptr;
      const float* dptr = has_dims ? dims : nullptr;
      const float* tptr = has_tau ? tau : nullptr;
      LaunchCfg gf = pick_cfg(ctx, 0, (int)n, params.flags);
      const size_t t0 = n - nb;  // the adjoint requests: a contiguous tail, recorded by the forward
      StepExtras fwd_rec, bwd_rec;
      fwd_rec.saved = nb ? saved : nullptr;
      fwd_rec.saved_stride = rs;
      fwd_rec.saved_first = (int32_t)t0;
      bwd_rec.saved = saved;
      bwd_rec.saved_stride = rs;
      st = enqueue_step(ctx, 0, gf, (int)n, pg, poses, dptr, tptr, &params, out, nullptr, nullptr, nullptr, scratch,
                        order, counter, s, b->max_ee, fwd_rec);
      if (st == CM_OK && nb) {
        LaunchCfg gb = pick_cfg(ctx, 1, (int)nb, params.flags);
        st = enqueue_step(ctx, 1, gb, (int)nb, pg + 2 * t0, poses + 14 * t0, has_dims ? dims + 6 * t0 : nullptr,
                          has_tau ? tau + t0 : nullptr, &params, nullptr, gout, gp, gd, scratch, order, counter, s,
                          b->max_ee, bwd_rec);
      }
    }
    if (st != CM_OK) return st;
    // outputs
    off = offb = 0;
    for (Request* r : b->reqs) {
      const size_t m = (size_t)r->d.n_pairs;
      cudaMemcpyAsync(r->d.out, out + (size_t)8 * K * off, 32 * K * m, cudaMemcpyDeviceToHost, s);
      if (r->d.with_backward) {
        cudaMemcpyAsync(r->d.grad_poses, gp + 14 * offb, 56 * m, cudaMemcpyDeviceToHost, s);
        if (r->d.grad_dims) cudaMemcpyAsync(r->d.grad_dims, gd + 6 * offb, 24 * m, cudaMemcpyDeviceToHost, s);
        offb += m;
      }
      off += m;
    }
    if ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "batch event");
    if ((e = cudaEventRecord(b->done, s)) != cudaSuccess) return cuda_fail(e, "batch event");
    return CM_OK;
  }

  void loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      retire_finished(lk);
      if (stop && queue.empty() && running.empty()) break;
      std::unique_ptr<Batch> b = form_batch();
      if (b) {
        for (Request* r : b->reqs) r->state = 1;
        lk.unlock();
        cm_status st = issue(b.get());
        lk.lock();
        if (st != CM_OK) {
          for (Request* r : b->reqs) {
            r->state = 3;
            r->status = st;
            r->t_done = Clock::now();
          }
          bytes_in_use -= b->bytes;
          for (size_t s = 0; s < streams.size(); ++s)
            if (streams[s] == b->stream) stream_busy[s] = 0;
          if (b->done) cudaEventDestroy(b->done);
          if (b->mem) cudaFreeAsync(b->mem, b->stream);
          cv_done.notify_all();
        } else {
          running.push_back(std::move(b));
        }
        continue;
      }
      // nothing to issue: wait for a submission, or poll the running batches
      if (running.empty())
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      else
        cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
};

}  // namespace cm

cm_context::cm_context() = default;
cm_context::~cm_context() = default;

void cm::rt::server_shutdown(cm_context* c) { c->server.reset(); }

extern "C" {

cm_status cm_server_start(cm_context* c, const cm_params* params, int32_t max_batch_pairs, int32_t n_streams) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  cm_status st = check_params(params);
  if (st != CM_OK) return st;
  if (max_batch_pairs <= 0 || n_streams <= 0 || n_streams > 16)
    return fail(CM_ERR_INVALID_ARG, "max_batch_pairs must be > 0 and n_streams in 1..16");
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->server) return fail(CM_ERR_INVALID_ARG, "server already running");
  if (c->hdr.empty()) return fail(CM_ERR_INVALID_ARG, "register geometry before starting the server");
  if ((st = check_k(c, params)) != CM_OK) return st;
  cudaSetDevice(c->device);
  if ((st = sync_geometry_locked(c)) != CM_OK) return st;
  auto srv = std::make_unique<Server>();
  srv->ctx = c;
  srv->params = *params;
  srv->max_batch_pairs = max_batch_pairs;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "server stream");
    srv->streams.push_back(s);
    srv->stream_busy.push_back(0);
  }
  // the most CTAs any launch shape of a batch may use (scratch slices per batch)
  int gmax = 1;
  for (int blk : {64, 128, 256, 512}) {
    SmemLayout L;
    int g = 1;
    shape(c, 0, LaunchCfg{blk, 0, 1}, max_batch_pairs, L, g);
    gmax = std::max(gmax, g);
    if (blk >= 128 && blk <= 256) {  // the adjoint's shapes
      for (int ps : {1, 2}) {
        shape(c, 1, LaunchCfg{blk, ps, 1}, max_batch_pairs, L, g);
        gmax = std::max(gmax, g);
      }
    }
  }
  srv->grid_max = gmax;
  if (c->budget && srv->batch_bytes(1, 1, 1) > c->budget)
    return fail(CM_ERR_ADMISSION, "the HBM budget does not even hold a one-pair batch");
  // batch memory comes from the server's own stream-ordered pool, which keeps freed
  // blocks cached (up to the budget) instead of returning them to the driver
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = c->device;
  cudaError_t pe = cudaMemPoolCreate(&srv->mempool, &props);
  if (pe != cudaSuccess) {
    srv->mempool = nullptr;
    return cuda_fail(pe, "server memory pool");
  }
  uint64_t keep = c->budget ? (uint64_t)c->budget : UINT64_MAX;
  cudaMemPoolSetAttribute(srv->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
  Server* raw = srv.get();
  c->server = std::move(srv);
  raw->thread = std::thread([raw] { raw->loop(); });
  return CM_OK;
}

cm_status cm_submit(cm_context* c, const cm_request_desc* d, uint64_t* ticket) {
  if (!c || !d || !ticket) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  Server* s = c->server.get();
  if (!s) return fail(CM_ERR_INVALID_ARG, "server not started");
  if (d->n_pairs <= 0 || d->n_pairs > s->max_batch_pairs)
    return fail(CM_ERR_INVALID_ARG, "n_pairs must be in 1..max_batch_pairs");
  if (!d->pair_geoms || !d->poses || !d->out) return fail(CM_ERR_INVALID_ARG, "pair_geoms, poses and out are required");
  if (d->with_backward && (!d->grad_out || !d->grad_poses))
    return fail(CM_ERR_INVALID_ARG, "a backward request needs grad_out and grad_poses");
  auto r = std::make_unique<Request>();
  r->d = *d;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    const int ng = (int)c->hdr.size();
    int64_t m = 1;
    for (int i = 0; i < d->n_pairs; ++i) {
      const int a = d->pair_geoms[2 * i], b = d->pair_geoms[2 * i + 1];
      if (a >= 0 && a < ng && b >= 0 && b < ng)
        m = std::max<int64_t>(m, (int64_t)c->hdr[a].n_edges * c->hdr[b].n_edges);
    }
    r->max_ee = m;
  }
  if (s->batch_bytes(d->n_pairs, d->with_backward ? d->n_pairs : 0, r->max_ee) > s->budget())
    return fail(CM_ERR_ADMISSION, "request does not fit the HBM budget even alone");
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->reqs.empty() || !s->queue.empty()) {
      // dims / tau are either given by every request or by none (one batch, one layout)
      const Request* any = s->reqs.begin()->second.get();
      if ((any->d.dims == nullptr) != (d->dims == nullptr) || (any->d.tau == nullptr) != (d->tau == nullptr))
        return fail(CM_ERR_INVALID_ARG, "all requests of a server must agree on giving dims and tau");
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
  }
  s->cv_work.notify_one();
  return CM_OK;
}

cm_status cm_poll(cm_context* c, uint64_t ticket, int32_t* done) {
  if (!c || !done) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  Server* s = c->server.get();
  if (!s) return fail(CM_ERR_INVALID_ARG, "server not started");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(CM_ERR_NOT_FOUND, "unknown ticket");
  *done = it->second->state >= 2 ? 1 : 0;
  return it->second->state == 3 ? it->second->status : CM_OK;
}

cm_status cm_wait(cm_context* c, uint64_t ticket, int32_t timeout_ms) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  Server* s = c->server.get();
  if (!s) return fail(CM_ERR_INVALID_ARG, "server not started");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(CM_ERR_NOT_FOUND, "unknown ticket");
  Request* r = it->second.get();
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  while (r->state < 2) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2)
      return fail(CM_ERR_TIMEOUT, "request not finished before the deadline");
  }
  if (r->state == 3)
    return fail(r->status, r->status == CM_ERR_ADMISSION ? "request does not fit the device's free memory"
                                                         : "request failed on the device");
  return CM_OK;
}

cm_status cm_request_latency(cm_context* c, uint64_t ticket, double* seconds) {
  if (!c || !seconds) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  Server* s = c->server.get();
  if (!s) return fail(CM_ERR_INVALID_ARG, "server not started");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(CM_ERR_NOT_FOUND, "unknown ticket");
  if (it->second->state < 2) return fail(CM_ERR_TIMEOUT, "request not finished");
  *seconds = std::chrono::duration<double>(it->second->t_done - it->second->t_submit).count();
  return CM_OK;
}

cm_status cm_release(cm_context* c, uint64_t ticket) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  Server* s = c->server.get();
  if (!s) return fail(CM_ERR_INVALID_ARG, "server not started");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(CM_ERR_NOT_FOUND, "unknown ticket");
  if (it->second->state < 2) return fail(CM_ERR_INVALID_ARG, "request still in flight");
  s->reqs.erase(it);
  return CM_OK;
}

cm_status cm_server_stats(cm_context* c, uint64_t* pairs_done, uint64_t* batches_done, uint64_t* bytes_in_use) {
  if (!c || !pairs_done || !batches_done || !bytes_in_use) return fail(CM_ERR_INVALID_ARG, "NULL argument");
  Server* s = c->server.get();
  if (!s) return fail(CM_ERR_INVALID_ARG, "server not started");
  std::lock_guard<std::mutex> lk(s->mu);
  *pairs_done = s->pairs_done;
  *batches_done = s->batches_done;
  *bytes_in_use = s->bytes_in_use;
  return CM_OK;
}

cm_status cm_server_stop(cm_context* c) {
  if (!c) return fail(CM_ERR_INVALID_ARG, "NULL context");
  c->server.reset();  // drains the queue, waits for running batches
  return CM_OK;
}

}  // extern "C"
