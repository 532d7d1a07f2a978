// Native continuous-batching query loop for trained fields (the serving form of the forward
// path, Sec. 5 a-d then the network): one scheduler thread merges queued requests of the same
// dimension into batches, admits a batch when its buffers fit in the caller's device arena next
// to the batches in flight, and runs each batch on its own stream slot -- host-to-device copies
// of its requests' points, encode_fwd, mlp_fwd, device-to-host copies of the values -- ending in
// a host callback that completes its requests.  No device memory is allocated here.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <exception>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "sxe_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int64_t kAlign = 256;
constexpr int kMaxSlots = 16;
constexpr size_t kCopyPiece = (size_t)4 << 20;   // bytes per copy command

int64_t align_up(int64_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
int64_t dtype_bytes(int32_t dt) { return dt == SXE_F32 ? 4 : 2; }

struct SrvField {
  const sxe_encoder* enc = nullptr;
  const void* tables = nullptr;
  sxe_mlp_desc mlp{};
  const void* weights = nullptr;
};

struct SrvRequest {
  int64_t id = 0;
  int d = 0;
  const float* x = nullptr;
  float* y = nullptr;
  int64_t n = 0;
  Clock::time_point t_arrival, t_done;
  int state = 0;                 // 0 pending, 1 done, 2 failed
  std::string error;
};

struct SrvBatch;

}  // namespace

struct sxe_server {
  sxe_server_desc desc{};
  int device = 0;
  SrvField fields[6];            // by d (2..5)
  cudaStream_t streams[kMaxSlots] = {};      // normal priority
  cudaStream_t streams_hi[kMaxSlots] = {};   // high priority (small batches)
  std::vector<int> free_slots;
  std::deque<SrvRequest*> queue;
  std::unordered_map<int64_t, std::unique_ptr<SrvRequest>> requests;
  std::vector<std::pair<int64_t, int64_t>> used;   // arena ranges [begin, end) of batches in flight
  int64_t used_bytes = 0, peak_bytes = 0, n_batches = 0, next_id = 0;
  int inflight = 0;
  bool running = false, stopping = false, drain = true;
  std::mutex mu;
  std::mutex stop_mu;            // serialises sxe_server_stop calls (one of them joins the thread)
  std::condition_variable cv_sched, cv_done;
  std::thread thread;
};

namespace {

struct SrvBatch {
  sxe_server* srv = nullptr;
  int slot = 0;
  cudaStream_t stream = nullptr;
  int64_t begin = 0, end = 0;
  std::vector<SrvRequest*> reqs;
};

// Arena bytes of a batch of P points of field f: points, encoding, values, each 256-aligned.
int64_t batch_bytes(const SrvField& f, int64_t P) {
  const int d = f.enc->desc.d;
  const int64_t n_enc = (int64_t)f.enc->desc.n_levels * f.enc->desc.n_features;
  return align_up(P * d * 4) + align_up(P * n_enc * dtype_bytes(f.enc->desc.out_dtype)) +
         align_up(P * (int64_t)f.mlp.n_out * 4);
}

// First free range of `bytes` in the arena next to the ranges in use (sorted), or -1.
int64_t find_range(const sxe_server* s, int64_t bytes) {
  int64_t at = 0;
  for (const auto& r : s->used) {
    if (r.first - at >= bytes) return at;
    at = std::max(at, r.second);
  }
  return s->desc.arena_bytes - at >= bytes ? at : -1;
}

void release_range(sxe_server* s, int64_t begin) {
  for (size_t i = 0; i < s->used.size(); ++i)
    if (s->used[i].first == begin) {
      s->used_bytes -= s->used[i].second - s->used[i].first;
      s->used.erase(s->used.begin() + (long)i);
      return;
    }
}

void finish(sxe_server* s, SrvBatch* b, int state, const std::string& err) {
  const auto now = Clock::now();
  for (SrvRequest* r : b->reqs) {
    r->t_done = now;
    r->state = state;
    if (state == 2) r->error = err;
  }
  release_range(s, b->begin);
  s->free_slots.push_back(b->slot);
  --s->inflight;
}

// Host callback at the end of a batch's stream work (run on a CUDA runtime thread; no CUDA calls here).
// Everything happens under the lock, so that once it is released the server may be destroyed.
void CUDART_CB batch_done(void* p) {
  SrvBatch* b = static_cast<SrvBatch*>(p);
  sxe_server* s = b->srv;
  std::lock_guard<std::mutex> lock(s->mu);
  finish(s, b, 1, std::string());
  delete b;
  s->cv_done.notify_all();
  s->cv_sched.notify_all();
}

}  // namespace

namespace {

// Enqueues one batch on its slot's stream; returns an error text, empty on success (the host
// callback then completes the batch).
std::string launch_batch(sxe_server* s, const SrvField& f, SrvBatch* b, int64_t P) {
  cudaStream_t st = b->stream;
  const int d = f.enc->desc.d;
  const int64_t n_enc = (int64_t)f.enc->desc.n_levels * f.enc->desc.n_features;
  const int n_out = f.mlp.n_out;
  unsigned char* base = static_cast<unsigned char*>(s->desc.arena) + b->begin;
  float* x = reinterpret_cast<float*>(base);
  void* enc = base + align_up(P * d * 4);
  float* y = reinterpret_cast<float*>(base + align_up(P * d * 4) + align_up(P * n_enc * dtype_bytes(f.enc->desc.out_dtype)));
  int64_t o = 0;
  for (SrvRequest* r : b->reqs) {
    // in pieces of at most kCopyPiece bytes (the values too, below), so that a small batch's
    // copies on another stream are served between the pieces of a large one's
    const size_t total = (size_t)(r->n * d) * sizeof(float);
    for (size_t at = 0; at < total; at += kCopyPiece) {
      const size_t len = std::min(kCopyPiece, total - at);
      const cudaError_t e = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(x + o * d) + at,
                                            reinterpret_cast<const unsigned char*>(r->x) + at, len,
                                            cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return std::string("points copy: ") + cudaGetErrorString(e);
    }
    o += r->n;
  }
  if (sxe::launch_encode_fwd(f.enc, x, P, f.tables, enc, st) != SXE_OK) return sxe_last_error();
  if (sxe::launch_mlp_fwd(&f.mlp, f.weights, enc, P, y, nullptr, st, true) != SXE_OK) return sxe_last_error();
  o = 0;
  for (SrvRequest* r : b->reqs) {
    const size_t total = (size_t)(r->n * n_out) * sizeof(float);
    for (size_t at = 0; at < total; at += kCopyPiece) {
      const size_t len = std::min(kCopyPiece, total - at);
      const cudaError_t e = cudaMemcpyAsync(reinterpret_cast<unsigned char*>(r->y) + at,
                                            reinterpret_cast<const unsigned char*>(y + o * n_out) + at, len,
                                            cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return std::string("values copy: ") + cudaGetErrorString(e);
    }
    o += r->n;
  }
  const cudaError_t e = cudaLaunchHostFunc(st, batch_done, b);
  if (e != cudaSuccess) return std::string("completion callback: ") + cudaGetErrorString(e);
  return std::string();
}

void serve_loop(sxe_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  auto leaving = [s] { return s->stopping && (!s->drain || s->queue.empty()); };
  for (;;) {
    s->cv_sched.wait(lk, [&] { return leaving() || (!s->queue.empty() && !s->free_slots.empty()); });
    if (leaving()) break;
    // the head request and the later queued requests of its d and its size class, in arrival
    // order, up to the class's batch limit (small requests, of at most priority_points points,
    // form high-priority batches of at most that size and are not merged into large batches);
    // shrunk from the back until the batch fits in the arena beside those in flight
    SrvRequest* head = s->queue.front();
    const SrvField& f = s->fields[head->d];
    const bool small = head->n <= s->desc.priority_points;
    const int64_t limit = small ? std::min(s->desc.priority_points, s->desc.max_batch_points) : s->desc.max_batch_points;
    std::vector<SrvRequest*> group;
    int64_t P = 0;
    for (SrvRequest* r : s->queue)
      if (r->d == head->d && (r->n <= s->desc.priority_points) == small && P + r->n <= limit) {
        group.push_back(r);
        P += r->n;
      }
    int64_t bytes = batch_bytes(f, P), at = find_range(s, bytes);
    while (at < 0 && group.size() > 1) {
      P -= group.back()->n;
      group.pop_back();
      bytes = batch_bytes(f, P);
      at = find_range(s, bytes);
    }
    if (at < 0) {                       // wait for a batch in flight to free its range
      const int before = s->inflight;
      s->cv_sched.wait(lk, [&] { return s->inflight < before || leaving(); });
      continue;
    }
    for (SrvRequest* r : group) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    SrvBatch* b = new SrvBatch;
    b->srv = s;
    b->slot = s->free_slots.back();
    s->free_slots.pop_back();
    b->stream = P <= s->desc.priority_points ? s->streams_hi[b->slot] : s->streams[b->slot];
    b->begin = at;
    b->end = at + bytes;
    b->reqs = std::move(group);
    s->used.emplace_back(at, at + bytes);
    std::sort(s->used.begin(), s->used.end());
    s->used_bytes += bytes;
    s->peak_bytes = std::max(s->peak_bytes, s->used_bytes);
    ++s->inflight;
    ++s->n_batches;
    lk.unlock();
    const std::string err = launch_batch(s, f, b, P);
    if (!err.empty()) cudaStreamSynchronize(b->stream);   // what was enqueued has run
    lk.lock();
    if (!err.empty()) {
      finish(s, b, 2, err);
      delete b;
      s->cv_done.notify_all();
    }
  }
  const auto now = Clock::now();
  for (SrvRequest* r : s->queue) {     // not draining: what is still queued fails
    r->state = 2;
    r->error = "server stopped before the request ran";
    r->t_done = now;
  }
  s->queue.clear();
  s->cv_done.notify_all();
  s->cv_sched.wait(lk, [&] { return s->inflight == 0; });
}

bool is_aligned(const void* p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

extern "C" {

sxe_status sxe_server_create(const sxe_server_desc* desc, sxe_server** out) {
  using sxe::set_error;
  if (!desc || !out) return set_error(SXE_EINVAL, "server_create: NULL desc or out");
  if (!desc->arena || !is_aligned(desc->arena, kAlign) || desc->arena_bytes <= 0)
    return set_error(SXE_EINVAL, "server_create: the arena must be a non-empty 256-byte aligned device buffer");
  if (desc->n_slots < 1 || desc->n_slots > kMaxSlots)
    return set_error(SXE_EINVAL, "server_create: n_slots=%d outside 1..%d", desc->n_slots, kMaxSlots);
  if (desc->max_batch_points < 1) return set_error(SXE_EINVAL, "server_create: max_batch_points < 1");
  if (desc->priority_points < 0) return set_error(SXE_EINVAL, "server_create: priority_points < 0");
  std::unique_ptr<sxe_server> s(new sxe_server);
  s->desc = *desc;
  int lo = 0, hi = 0;
  if (cudaGetDevice(&s->device) != cudaSuccess || cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess)
    return sxe::check_launch("server_create");
  for (int i = 0; i < desc->n_slots; ++i) {
    cudaError_t e = cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->streams_hi[i], cudaStreamNonBlocking, hi);
    if (e != cudaSuccess) {
      for (int j = 0; j <= i; ++j) {
        if (s->streams[j]) cudaStreamDestroy(s->streams[j]);
        if (s->streams_hi[j]) cudaStreamDestroy(s->streams_hi[j]);
      }
      return set_error(SXE_ECUDA, "server_create: %s", cudaGetErrorString(e));
    }
    s->free_slots.push_back(desc->n_slots - 1 - i);
  }
  *out = s.release();
  return SXE_OK;
}

sxe_status sxe_server_add_field(sxe_server* s, const sxe_encoder* enc, const void* tables, const sxe_mlp_desc* mlp,
                                const void* weights) {
  using sxe::set_error;
  if (!s || !enc || !tables || !mlp || !weights) return set_error(SXE_EINVAL, "server_add_field: NULL argument");
  sxe_status st = sxe::check_mlp("server_add_field", mlp);
  if (st != SXE_OK) return st;
  const int d = enc->desc.d;
  if (d < 2 || d > 5) return set_error(SXE_EINVAL, "server_add_field: d=%d outside 2..5", d);
  if (enc->desc.out_dtype != mlp->dtype)
    return set_error(SXE_EINVAL, "server_add_field: the encoding's output type is not the network's dtype");
  if (enc->desc.n_levels * enc->desc.n_features != mlp->n_in)
    return set_error(SXE_EINVAL, "server_add_field: L*F=%d is not the network's n_in=%d",
                     enc->desc.n_levels * enc->desc.n_features, mlp->n_in);
  if (!is_aligned(weights, 4)) return set_error(SXE_EINVAL, "server_add_field: weights misaligned");
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->running) return set_error(SXE_EINVAL, "server_add_field: server already started");
  s->fields[d] = SrvField{enc, tables, *mlp, weights};
  return SXE_OK;
}

sxe_status sxe_server_start(sxe_server* s) {
  using sxe::set_error;
  if (!s) return set_error(SXE_EINVAL, "server_start: NULL server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->running) return set_error(SXE_EINVAL, "server_start: already running");
  bool any = false;
  for (int d = 2; d <= 5; ++d) any |= s->fields[d].enc != nullptr;
  if (!any) return set_error(SXE_EINVAL, "server_start: no field registered");
  s->running = true;
  s->stopping = false;
  try {
    s->thread = std::thread(serve_loop, s);
  } catch (const std::exception& e) {
    s->running = false;
    return set_error(SXE_ENOMEM, "server_start: no scheduler thread (%s)", e.what());
  }
  return SXE_OK;
}

sxe_status sxe_server_submit(sxe_server* s, int32_t d, const float* x, int64_t n, float* y, int64_t* request_id) {
  using sxe::set_error;
  if (!s || !x || !y || !request_id) return set_error(SXE_EINVAL, "server_submit: NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  if (!s->running || s->stopping) return set_error(SXE_EINVAL, "server_submit: server not running");
  if (d < 2 || d > 5 || !s->fields[d].enc) return set_error(SXE_EINVAL, "server_submit: no field of dimension %d", d);
  if (n < 1 || n > s->desc.max_batch_points)
    return set_error(SXE_EINVAL, "server_submit: %lld points outside 1..max_batch_points", (long long)n);
  if (batch_bytes(s->fields[d], n) > s->desc.arena_bytes)
    return set_error(SXE_EINVAL, "server_submit: %lld points need more than the arena", (long long)n);
  try {
    std::unique_ptr<SrvRequest> r(new SrvRequest);
    r->id = s->next_id;
    r->d = d;
    r->x = x;
    r->y = y;
    r->n = n;
    r->t_arrival = Clock::now();
    SrvRequest* q = r.get();
    s->requests.emplace(r->id, std::move(r));
    try {
      s->queue.push_back(q);
    } catch (...) {
      s->requests.erase(q->id);
      throw;
    }
    *request_id = s->next_id++;
  } catch (const std::exception& e) {
    return set_error(SXE_ENOMEM, "server_submit: %s", e.what());
  }
  lock.unlock();
  s->cv_sched.notify_all();
  return SXE_OK;
}

sxe_status sxe_server_wait(sxe_server* s, int64_t id, int64_t timeout_us, int32_t* state, double* latency_s) {
  using sxe::set_error;
  if (!s || !state) return set_error(SXE_EINVAL, "server_wait: NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->requests.find(id);
  if (it == s->requests.end()) return set_error(SXE_EINVAL, "server_wait: unknown request %lld", (long long)id);
  SrvRequest* r = it->second.get();
  if (r->state == 0 && timeout_us > 0)
    s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [r] { return r->state != 0; });
  *state = r->state;
  if (r->state == 0) return SXE_OK;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_arrival).count();
  const std::string err = r->error;
  s->requests.erase(it);
  if (*state == 2) set_error(SXE_ECUDA, "server request %lld failed: %s", (long long)id, err.c_str());
  return SXE_OK;
}

sxe_status sxe_server_stop(sxe_server* s, int32_t drain) {
  if (!s) return sxe::set_error(SXE_EINVAL, "server_stop: NULL server");
  std::lock_guard<std::mutex> one_stop(s->stop_mu);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->running) return SXE_OK;
    s->stopping = true;
    s->drain = drain != 0;
  }
  s->cv_sched.notify_all();
  s->thread.join();
  std::lock_guard<std::mutex> lock(s->mu);
  s->running = false;
  s->stopping = false;
  return SXE_OK;
}

sxe_status sxe_server_stats(const sxe_server* s, int64_t* n_batches, int64_t* peak_bytes) {
  if (!s) return sxe::set_error(SXE_EINVAL, "server_stats: NULL server");
  sxe_server* m = const_cast<sxe_server*>(s);
  std::lock_guard<std::mutex> lock(m->mu);
  if (n_batches) *n_batches = s->n_batches;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  return SXE_OK;
}

sxe_status sxe_server_destroy(sxe_server* s) {
  if (!s) return SXE_OK;
  sxe_server_stop(s, 1);
  for (int i = 0; i < s->desc.n_slots; ++i) {
    cudaStreamSynchronize(s->streams[i]);
    cudaStreamSynchronize(s->streams_hi[i]);
    cudaStreamDestroy(s->streams[i]);
    cudaStreamDestroy(s->streams_hi[i]);
  }
  delete s;
  return SXE_OK;
}

}  // extern "C"
