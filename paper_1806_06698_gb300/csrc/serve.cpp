// serve.cpp -- continuous-batching request server around the batched
// eigensolver (host runtime of libsyev3; no kernel of its own).
//
// Requests reference device-resident packed matrices (FP64 or FP32) and get
// their eigenvalues / eigenvectors in a device arena of fixed size (the
// memory budget), allocated once at creation.  A dispatcher thread
//  * admits waiting requests in arrival order as soon as the arena has room
//    for their outputs (a request larger than the whole arena is refused at
//    submission);
//  * cuts admitted requests into chunks and issues them round-robin across
//    all admitted requests onto a set of CUDA streams, at most
//    `max_inflight` chunks per stream, so a small request that arrives
//    behind a large one is on the device after at most one chunk per
//    stream, and the work of different requests overlaps on the device;
//  * learns of finished chunks from host functions enqueued behind them
//    (cudaLaunchHostFunc), which only touch host state.
// Results stay in the arena until the client releases the request.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/syev3.h"

namespace {

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing on free.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    free_[0] = size;
    size_ = size;
    used_ = 0;
    peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t size() const { return size_; }
  static constexpr size_t kAlign = 256;

 private:
  std::map<size_t, size_t> free_;  // offset -> length
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

struct Request {
  uint64_t ticket;
  int dtype;
  const char* A;
  int64_t n;
  bool vectors;
  size_t es;
  size_t out_off = 0, out_bytes = 0;
  char* lam = nullptr;
  char* U = nullptr;
  int64_t next = 0;       // first matrix not yet issued
  int64_t finished = 0;   // matrices whose chunk completed
  int state = 0;          // 0 waiting, 1 admitted, 2 done, 3 failed
  int64_t t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct syev3_server_s;

namespace {

struct ChunkDone {
  syev3_server_s* srv;
  uint64_t ticket;
  int64_t count;
  int stream;
};

}  // namespace

struct syev3_server_s {
  syev3_server_config cfg;
  int device = 0;
  char* arena_base = nullptr;
  Arena arena;
  std::vector<cudaStream_t> streams;
  std::vector<int> inflight;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> waiting;
  std::vector<uint64_t> active;  // admitted, with matrices left to issue
  size_t rr = 0;                 // round-robin cursor over active
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  int error = SYEV3_OK;
  int64_t completed = 0, matrices_done = 0, chunks_issued = 0;
  std::thread dispatcher;

  void run();
};

namespace {

void CUDART_CB on_chunk_done(void* p) {
  std::unique_ptr<ChunkDone> c(static_cast<ChunkDone*>(p));
  syev3_server_s* s = c->srv;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->inflight[c->stream]--;
    auto it = s->reqs.find(c->ticket);
    if (it != s->reqs.end()) {
      Request& r = *it->second;
      r.finished += c->count;
      if (r.finished == r.n && r.state == 1) {
        r.state = 2;
        r.t_done = now_ns();
        s->completed++;
        s->matrices_done += r.n;
      }
    }
  }
  s->cv.notify_all();
}

}  // namespace

void syev3_server_s::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    bool progress = false;
    // Admission: arrival order, as far as the arena has room.
    while (!waiting.empty()) {
      Request& r = *reqs[waiting.front()];
      size_t off;
      if (!arena.alloc(r.out_bytes, &off)) break;
      r.out_off = off;
      r.lam = arena_base + off;
      r.U = r.vectors ? r.lam + ((r.n * 3 * r.es + 255) / 256 * 256) : nullptr;
      r.state = 1;
      r.t_admit = now_ns();
      active.push_back(r.ticket);
      waiting.pop_front();
      progress = true;
    }
    // Issue: round-robin over admitted requests, one chunk at a time, onto
    // any stream with room.
    for (size_t s = 0; s < streams.size() && !active.empty(); ++s) {
      while (inflight[s] < cfg.max_inflight && !active.empty()) {
        if (rr >= active.size()) rr = 0;
        Request& r = *reqs[active[rr]];
        const int64_t cnt = std::min<int64_t>(cfg.chunk, r.n - r.next);
        const int64_t b = r.next;
        r.next += cnt;
        const bool last = (r.next == r.n);
        if (last) {
          active.erase(active.begin() + rr);
        } else {
          ++rr;
        }
        inflight[s]++;
        chunks_issued++;
        lk.unlock();
        int st = syev3_batched(r.A + b * 6 * r.es, cnt, r.lam + b * 3 * r.es, r.U ? r.U + b * 9 * r.es : nullptr,
                               r.dtype, reinterpret_cast<syev3_stream_t>(streams[s]));
        cudaError_t e = cudaSuccess;
        if (st == SYEV3_OK) {
          auto* c = new ChunkDone{this, r.ticket, cnt, (int)s};
          e = cudaLaunchHostFunc(streams[s], on_chunk_done, c);
          if (e != cudaSuccess) delete c;
        }
        lk.lock();
        if (st != SYEV3_OK || e != cudaSuccess) {
          inflight[s]--;
          r.state = 3;
          error = (st != SYEV3_OK) ? st : SYEV3_ECUDA;
          active.erase(std::remove(active.begin(), active.end(), r.ticket), active.end());
        }
        progress = true;
      }
    }
    if (!progress) cv.wait_for(lk, std::chrono::milliseconds(5));
  }
}

extern "C" {

int syev3_server_create(const syev3_server_config* cfg, syev3_server** out) {
  if (out == nullptr) return SYEV3_EINVAL;
  syev3_server_config c;
  c.memory_budget_bytes = (size_t)16 << 30;
  c.num_streams = 4;
  c.chunk = (int64_t)1 << 18;
  c.max_inflight = 2;
  if (cfg) {
    if (cfg->memory_budget_bytes) c.memory_budget_bytes = cfg->memory_budget_bytes;
    if (cfg->num_streams > 0) c.num_streams = cfg->num_streams;
    if (cfg->chunk > 0) c.chunk = cfg->chunk;
    if (cfg->max_inflight > 0) c.max_inflight = cfg->max_inflight;
  }
  if (c.num_streams > 64 || c.chunk < 1) return SYEV3_EINVAL;
  auto s = std::make_unique<syev3_server_s>();
  s->cfg = c;
  if (cudaGetDevice(&s->device) != cudaSuccess) return SYEV3_ECUDA;
  if (cudaMalloc(&s->arena_base, c.memory_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    return SYEV3_ECUDA;
  }
  s->arena.reset(c.memory_budget_bytes);
  s->streams.resize(c.num_streams);
  s->inflight.assign(c.num_streams, 0);
  for (auto& st : s->streams)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SYEV3_ECUDA;
  syev3_server_s* raw = s.release();
  raw->dispatcher = std::thread([raw] { raw->run(); });
  *out = raw;
  return SYEV3_OK;
}

int syev3_server_destroy(syev3_server* srv) {
  if (srv == nullptr) return SYEV3_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  srv->dispatcher.join();
  for (auto& st : srv->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(srv->arena_base);
  delete srv;
  return SYEV3_OK;
}

int syev3_server_submit(syev3_server* srv, int dtype, const void* d_A, int64_t n, int vectors, uint64_t* ticket) {
  if (srv == nullptr || ticket == nullptr || d_A == nullptr || n <= 0) return SYEV3_EINVAL;
  if (dtype != SYEV3_F64 && dtype != SYEV3_F32 && dtype != SYEV3_F32_COMPENSATED) return SYEV3_EINVAL;
  auto r = std::make_unique<Request>();
  r->dtype = dtype;
  r->A = static_cast<const char*>(d_A);
  r->n = n;
  r->vectors = vectors != 0;
  r->es = dtype == SYEV3_F64 ? 8 : 4;
  r->out_bytes = (n * 3 * r->es + 255) / 256 * 256 + (r->vectors ? n * 9 * r->es : 0);
  if (r->out_bytes > srv->arena.size()) return SYEV3_EINVAL;  // can never be admitted
  r->t_submit = now_ns();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    r->ticket = srv->next_ticket++;
    *ticket = r->ticket;
    srv->waiting.push_back(r->ticket);
    srv->reqs.emplace(r->ticket, std::move(r));
  }
  srv->cv.notify_all();
  return SYEV3_OK;
}

int syev3_server_query(syev3_server* srv, uint64_t ticket, syev3_request_info* info) {
  if (srv == nullptr || info == nullptr) return SYEV3_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return SYEV3_EINVAL;
  const Request& r = *it->second;
  info->state = r.state;
  info->n = r.n;
  info->dtype = r.dtype;
  info->d_lambda = r.lam;
  info->d_U = r.U;
  info->t_submit_ns = r.t_submit;
  info->t_admit_ns = r.t_admit;
  info->t_done_ns = r.t_done;
  return SYEV3_OK;
}

int syev3_server_wait(syev3_server* srv, uint64_t ticket, double timeout_s) {
  if (srv == nullptr) return SYEV3_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return SYEV3_EINVAL;
  Request* r = it->second.get();
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  while (r->state < 2) {
    if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2) return SYEV3_ETIMEOUT;
  }
  return r->state == 2 ? SYEV3_OK : srv->error;
}

int syev3_server_release(syev3_server* srv, uint64_t ticket) {
  if (srv == nullptr) return SYEV3_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end() || it->second->state < 2) return SYEV3_EINVAL;
    if (it->second->lam) srv->arena.release(it->second->out_off, it->second->out_bytes);
    srv->reqs.erase(it);
  }
  srv->cv.notify_all();
  return SYEV3_OK;
}

int syev3_server_get_stats(syev3_server* srv, syev3_server_stats* st) {
  if (srv == nullptr || st == nullptr) return SYEV3_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  st->completed = srv->completed;
  st->matrices = srv->matrices_done;
  st->chunks = srv->chunks_issued;
  st->waiting = (int64_t)srv->waiting.size();
  st->arena_bytes = srv->arena.size();
  st->arena_used = srv->arena.used();
  st->arena_peak = srv->arena.peak();
  st->error = srv->error;
  return SYEV3_OK;
}

}  // extern "C"
