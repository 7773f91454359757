// Request server with continuous batching (the serving form of the pass; the paper's stated use
// is generating synthetic training images, Sec. 8.1).
//
// A scheduler thread owns admission.  Requests queue in arrival order; whenever a slot is free
// and the device-memory arena (one allocation of `memory_budget` bytes, first-fit with
// coalescing, bookkept on the host) can hold a request's buffers, the head request is admitted:
// its G-buffer is copied in as chunks spread over the server's copy streams (one host-to-device
// copy on one stream moves a fraction of what the host link carries; several in parallel fill
// it), its lights are copied and SSAO + blur + compose + tone map enqueued on one of the server's
// compute streams, which waits for the chunks, and the 8-bit image is copied out on it, so
// admitted requests overlap on the device.  A host-function callback at the end of each request's stream work stamps its
// completion and wakes the scheduler, which returns the memory and admits more.  Queued requests
// whose deadline passes are cancelled on the host (EPBR_ERR_TIMEOUT); nothing waits on the GPU
// without a bound.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "epbr_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;
constexpr int kCopyStreams = 4;                  // G-buffer upload streams
constexpr size_t kUploadChunk = (size_t)8 << 20;  // bytes per upload copy

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing of freed ranges.
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t n) {
    size = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        size_t rest = it->second - n, at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Device buffers of one request inside the arena.
struct Layout {
  size_t rt[4], lights, ao_raw, ao, ldr, total;
  int bpp[4];
};

Layout layout_of(const epbr_request& r) {
  Layout L;
  memset(&L, 0, sizeof(L));
  const int fp32[4] = {16, 16, 0, 4}, compact[4] = {4, 4, 2, 4};
  const int* b = r.format == EPBR_GBUFFER_FP32 ? fp32 : compact;
  size_t px = (size_t)r.width * r.height, ao = (size_t)((r.width + 1) / 2) * ((r.height + 1) / 2);
  size_t off = 0;
  for (int i = 0; i < 4; ++i) {
    L.bpp[i] = b[i];
    L.rt[i] = off;
    off += up(px * b[i]);
  }
  L.lights = off;
  off += up((size_t)r.num_lights * sizeof(epbr_light) + 16);
  L.ao_raw = off;
  off += up(ao * 4);
  L.ao = off;
  off += up(ao * 4);
  L.ldr = off;
  off += up(px * 4);
  L.total = off;
  return L;
}

struct Req {
  uint64_t id = 0;
  epbr_request r;
  Layout L;
  size_t off = 0;
  int stream = 0;
  bool deferred = false, done = false, admitted = false;
  Clock::time_point t_submit, t_admit, t_done;
  epbr_status status = EPBR_OK;
  std::string msg;
  void* server = nullptr;  // the epbr_server that owns it
};

}  // namespace

struct epbr_server {
  epbr_serve_config cfg;
  std::vector<epbr_ibl> ibls;
  int device = 0;
  char* d_arena = nullptr;
  Arena arena;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::vector<cudaStream_t> copy_streams;  // G-buffer uploads, chunk by chunk
  std::vector<cudaEvent_t> copy_events;    // one per copy stream: its latest chunk
  int next_copy = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> reqs;
  std::vector<Req*> finished;  // completed on the device, memory not yet returned
  int in_flight = 0;
  uint64_t next_id = 1;
  bool stop = false;
  epbr_serve_stats st;
  size_t bytes_in_use = 0;
  std::thread sched;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

void CUDART_CB on_device_done(void* p) {
  Req* q = (Req*)p;
  epbr_server* s = (epbr_server*)q->server;
  std::lock_guard<std::mutex> lk(s->mu);
  q->t_done = Clock::now();
  s->finished.push_back(q);
  s->cv_sched.notify_one();
}

// Called with the lock held.
void finish(epbr_server* s, Req* q, epbr_status status, const std::string& msg) {
  q->status = status;
  q->msg = msg;
  q->done = true;
  if (q->t_done == Clock::time_point()) q->t_done = Clock::now();
  if (status == EPBR_OK)
    s->st.completed++;
  else if (status == EPBR_ERR_TIMEOUT)
    s->st.timed_out++;
  else
    s->st.failed++;
  s->cv_done.notify_all();
}

// Enqueues a request's work on its stream (lock not held: only the scheduler touches q here).
epbr_status enqueue(epbr_server* s, Req* q) {
  const epbr_request& r = q->r;
  cudaStream_t st = s->streams[q->stream];
  char* base = s->d_arena + q->off;
  epbr_gbuffer g;
  memset(&g, 0, sizeof(g));
  g.format = r.format;
  g.width = r.width;
  g.height = r.height;
  for (int i = 0; i < 4; ++i) {
    if (!q->L.bpp[i]) continue;
    g.rt[i] = base + q->L.rt[i];
    g.pitch[i] = (int64_t)r.width * q->L.bpp[i];
    const size_t n = (size_t)r.width * r.height * q->L.bpp[i];
    // chunks of at most kUploadChunk bytes round-robin over the copy streams; the compute stream
    // waits for each (cudaStreamWaitEvent takes the event's latest record, so an event is free
    // for the next chunk of its stream as soon as the wait is enqueued)
    for (size_t o = 0; o < n; o += kUploadChunk) {
      const size_t c = n - o < kUploadChunk ? n - o : kUploadChunk;
      const int k = s->next_copy;
      s->next_copy = (s->next_copy + 1) % (int)s->copy_streams.size();
      if (cudaMemcpyAsync(base + q->L.rt[i] + o, (const char*)r.rt[i] + o, c, cudaMemcpyHostToDevice,
                          s->copy_streams[k]) != cudaSuccess ||
          cudaEventRecord(s->copy_events[k], s->copy_streams[k]) != cudaSuccess ||
          cudaStreamWaitEvent(st, s->copy_events[k], 0) != cudaSuccess)
        return epbr::fail(EPBR_ERR_CUDA, "serve: G-buffer upload: %s", cudaGetErrorString(cudaGetLastError()));
    }
  }
  epbr_light* d_lights = (epbr_light*)(base + q->L.lights);
  if (r.num_lights > 0 &&
      cudaMemcpyAsync(d_lights, r.lights, (size_t)r.num_lights * sizeof(epbr_light), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return epbr::fail(EPBR_ERR_CUDA, "serve: light upload: %s", cudaGetErrorString(cudaGetLastError()));
  int Wa = (r.width + 1) / 2;
  float* ao = (float*)(base + q->L.ao);
  epbr_status e = epbr_ssao(&g, &r.camera, &s->cfg.ssao, ao, (int64_t)Wa * 4, base + q->L.ao_raw,
                            q->L.ao - q->L.ao_raw, st);
  if (e) return e;
  epbr_shade_params sp;
  sp.flags = s->cfg.flags | EPBR_SHADE_EARLY_START;  // the kernel before it is the SSAO blur (or raw pass)
  sp.ao_scale = 2;
  sp.ao = ao;
  sp.ao_pitch = (int64_t)Wa * 4;
  uint8_t* ldr = (uint8_t*)(base + q->L.ldr);
  e = epbr_shade_tonemap(&g, &r.camera, d_lights, r.num_lights, &s->ibls[r.ibl_index], &sp, nullptr,
                         EPBR_HDR_RGBA32F, 0, &s->cfg.tonemap, ldr, (int64_t)r.width * 4, st);
  if (e) return e;
  if (cudaMemcpyAsync(r.ldr_out, ldr, (size_t)r.width * r.height * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return epbr::fail(EPBR_ERR_CUDA, "serve: result download: %s", cudaGetErrorString(cudaGetLastError()));
  if (cudaLaunchHostFunc(st, on_device_done, q) != cudaSuccess)
    return epbr::fail(EPBR_ERR_CUDA, "serve: completion callback: %s", cudaGetErrorString(cudaGetLastError()));
  return EPBR_OK;
}

void scheduler(epbr_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // 1. return the memory of requests the device has finished
    for (Req* q : s->finished) {
      s->arena.release(q->off, q->L.total);
      s->bytes_in_use -= q->L.total;
      s->in_flight--;
      finish(s, q, EPBR_OK, "");
    }
    s->finished.clear();
    // 2. cancel queued requests whose deadline passed (and everything queued on shutdown)
    Clock::time_point now = Clock::now();
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      Req* q = *it;
      bool late = q->r.deadline_ms > 0.0 && ms_between(q->t_submit, now) > q->r.deadline_ms;
      if (late || s->stop) {
        it = s->queue.erase(it);
        finish(s, q, EPBR_ERR_TIMEOUT, s->stop ? "server destroyed before admission" : "deadline passed in the queue");
      } else {
        ++it;
      }
    }
    if (s->stop && s->in_flight == 0) break;
    // 3. admit in arrival order while a slot and the memory are free
    while (!s->stop && !s->queue.empty() && s->in_flight < s->cfg.max_in_flight) {
      Req* q = s->queue.front();
      size_t off;
      if (!s->arena.alloc(q->L.total, &off)) {
        if (!q->deferred) s->st.deferred++;
        q->deferred = true;
        break;
      }
      s->queue.pop_front();
      q->off = off;
      q->stream = s->next_stream;
      s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
      q->admitted = true;
      q->t_admit = Clock::now();
      s->in_flight++;
      s->bytes_in_use += q->L.total;
      if (s->bytes_in_use > s->st.peak_bytes) s->st.peak_bytes = s->bytes_in_use;
      s->st.admitted++;
      lk.unlock();
      epbr_status e = enqueue(s, q);
      std::string msg = e ? epbr_last_error() : "";
      if (e) cudaStreamSynchronize(s->streams[q->stream]);  // nothing of it may still run
      lk.lock();
      if (e) {
        s->arena.release(q->off, q->L.total);
        s->bytes_in_use -= q->L.total;
        s->in_flight--;
        finish(s, q, e, msg);
      }
    }
    if (s->finished.empty()) {
      // sleep until a completion or a submission; wake periodically for deadlines
      s->cv_sched.wait_for(lk, std::chrono::milliseconds(1));
    }
  }
}

}  // namespace

using namespace epbr;

extern "C" epbr_status epbr_serve_create(const epbr_serve_config* cfg, epbr_server** out) {
  if (!cfg || !out) return fail(EPBR_ERR_INVALID_ARG, "serve: NULL argument");
  if (cfg->memory_budget < (1u << 20) || cfg->max_in_flight < 1 || cfg->num_streams < 1 || cfg->num_streams > 64 ||
      !cfg->ibls || cfg->num_ibls < 1)
    return fail(EPBR_ERR_INVALID_ARG, "serve: budget >= 1 MiB, max_in_flight >= 1, 1..64 streams, >= 1 ibl");
  if (cfg->ssao.scale != 2) return fail(EPBR_ERR_INVALID_ARG, "serve: ssao scale must be 2");
  epbr_server* s = new epbr_server();
  s->cfg = *cfg;
  s->ibls.assign(cfg->ibls, cfg->ibls + cfg->num_ibls);
  memset(&s->st, 0, sizeof(s->st));
  cudaGetDevice(&s->device);
  if (cudaMalloc(&s->d_arena, cfg->memory_budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail(EPBR_ERR_NO_MEMORY, "serve: arena of %zu bytes could not be allocated", cfg->memory_budget);
  }
  s->arena.init(cfg->memory_budget);
  for (int i = 0; i < cfg->num_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      cudaFree(s->d_arena);
      delete s;
      return fail(EPBR_ERR_CUDA, "serve: stream creation failed");
    }
    s->streams.push_back(st);
  }
  for (int i = 0; i < kCopyStreams; ++i) {
    cudaStream_t cs;
    cudaEvent_t ev;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      epbr_serve_destroy(s);
      return fail(EPBR_ERR_CUDA, "serve: copy stream creation failed");
    }
    s->copy_streams.push_back(cs);
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      epbr_serve_destroy(s);
      return fail(EPBR_ERR_CUDA, "serve: event creation failed");
    }
    s->copy_events.push_back(ev);
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return ok();
}

extern "C" epbr_status epbr_serve_request_bytes(const epbr_request* r, size_t* bytes) {
  if (!r || !bytes) return fail(EPBR_ERR_INVALID_ARG, "serve: NULL argument");
  if (r->format != EPBR_GBUFFER_FP32 && r->format != EPBR_GBUFFER_COMPACT)
    return fail(EPBR_ERR_INVALID_ARG, "serve: format");
  *bytes = layout_of(*r).total;
  return ok();
}

extern "C" epbr_status epbr_serve_submit(epbr_server* s, const epbr_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return fail(EPBR_ERR_INVALID_ARG, "serve: NULL argument");
  if (r->format != EPBR_GBUFFER_FP32 && r->format != EPBR_GBUFFER_COMPACT)
    return fail(EPBR_ERR_INVALID_ARG, "serve: G-buffer format %d", r->format);
  if (r->width < 1 || r->height < 1 || r->width > (1 << 15) || r->height > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "serve: size %dx%d", r->width, r->height);
  if (r->camera.width != r->width || r->camera.height != r->height || !(r->camera.fov_y > 0.0f))
    return fail(EPBR_ERR_INVALID_ARG, "serve: camera does not match the request");
  for (int i = 0; i < 4; ++i) {
    bool need = r->format == EPBR_GBUFFER_COMPACT || i != 2;
    if (need && !r->rt[i]) return fail(EPBR_ERR_INVALID_ARG, "serve: rt[%d] is NULL", i);
  }
  if (r->num_lights < 0 || r->num_lights > 65536 || (r->num_lights > 0 && !r->lights))
    return fail(EPBR_ERR_INVALID_ARG, "serve: lights");
  if (r->ibl_index < 0 || r->ibl_index >= (int)s->ibls.size()) return fail(EPBR_ERR_INVALID_ARG, "serve: ibl_index");
  if (!r->ldr_out) return fail(EPBR_ERR_INVALID_ARG, "serve: ldr_out is NULL");
  Req* q = new Req();
  q->r = *r;
  q->L = layout_of(*r);
  q->server = s;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete q;
    return fail(EPBR_ERR_INVALID_ARG, "serve: server is shutting down");
  }
  s->st.submitted++;
  if (q->L.total > s->cfg.memory_budget) {
    s->st.rejected++;
    size_t need = q->L.total;
    delete q;
    return fail(EPBR_ERR_ADMISSION, "serve: request needs %zu bytes, the budget is %zu", need, s->cfg.memory_budget);
  }
  q->id = s->next_id++;
  q->t_submit = Clock::now();
  s->queue.push_back(q);
  s->reqs[q->id] = q;
  *ticket = q->id;
  s->cv_sched.notify_one();
  return ok();
}

static void fill_result(const Req* q, epbr_result* out) {
  memset(out, 0, sizeof(*out));
  out->status = q->status;
  out->deferred = q->deferred ? 1 : 0;
  out->queue_ms = q->admitted ? ms_between(q->t_submit, q->t_admit) : ms_between(q->t_submit, q->t_done);
  out->latency_ms = ms_between(q->t_submit, q->t_done);
  strncpy(out->message, q->msg.c_str(), sizeof(out->message) - 1);
}

extern "C" epbr_status epbr_serve_wait(epbr_server* s, uint64_t ticket, int32_t timeout_ms, epbr_result* out) {
  if (!s || !out) return fail(EPBR_ERR_INVALID_ARG, "serve: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(EPBR_ERR_INVALID_ARG, "serve: unknown ticket %llu", (unsigned long long)ticket);
  Req* q = it->second;
  bool ok_ = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                 [&] { return q->done; });
  if (!ok_) return fail(EPBR_ERR_TIMEOUT, "serve: ticket %llu not done after %d ms", (unsigned long long)ticket,
                        timeout_ms);
  fill_result(q, out);
  s->reqs.erase(it);
  delete q;
  return ok();
}

extern "C" epbr_status epbr_serve_poll(epbr_server* s, uint64_t ticket, int32_t* done, epbr_result* out) {
  if (!s || !done || !out) return fail(EPBR_ERR_INVALID_ARG, "serve: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(EPBR_ERR_INVALID_ARG, "serve: unknown ticket %llu", (unsigned long long)ticket);
  Req* q = it->second;
  *done = q->done ? 1 : 0;
  if (q->done) {
    fill_result(q, out);
    s->reqs.erase(it);
    delete q;
  }
  return ok();
}

extern "C" epbr_status epbr_serve_get_stats(epbr_server* s, epbr_serve_stats* out) {
  if (!s || !out) return fail(EPBR_ERR_INVALID_ARG, "serve: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->in_flight = s->in_flight;
  out->queued = (int32_t)s->queue.size();
  out->bytes_in_use = s->bytes_in_use;
  return ok();
}

extern "C" epbr_status epbr_serve_destroy(epbr_server* s) {
  if (!s) return ok();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_sched.notify_one();
  }
  if (s->sched.joinable()) s->sched.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaStream_t st : s->copy_streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t ev : s->copy_events) cudaEventDestroy(ev);
  cudaFree(s->d_arena);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return ok();
}
