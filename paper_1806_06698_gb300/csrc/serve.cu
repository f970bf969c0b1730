// serve.cu -- the serving form of libsyev3: a continuous-batching request
// server whose queues, admission state and results live on the device (not
// in the paper, whose method each request's matrices run through).
//
// Device memory holds
//  * the request ring: one slot per outstanding request (kSlots), with its
//    input pointer, size, state, output extent and progress;
//  * the admission state: a FIFO over tickets and the arena of the memory
//    budget as a sorted list of free extents (first fit, coalescing);
//  * the work lists of the current round (ServeList, internal.h);
//  * the arena itself, which receives every request's eigenvalues and
//    eigenvectors and keeps them until the client releases the request.
// A round is five launches on the server's stream:
//  1. k_serve_admit (one CTA): takes the releases and new descriptors the
//     host passes as kernel arguments, frees and admits in arrival order as
//     far as the arena has room, and builds the round's work: up to `chunk`
//     matrices of every admitted request with work left (round-robin, at
//     most `round_matrices` in all), as one ragged list per element type;
//  2-4. the solve kernels' serving builds, each walking its list's tiles as
//     one batch (k_syev3_f64, k_syev3_f32 plain and compensated), so the
//     work of every admitted request shares each launch;
//  5. k_serve_complete (one CTA): adds the round's work to each request,
//     marks finished requests done with a device timestamp.
// Admissions and completions are published as records in a mailbox in
// mapped host memory; a host dispatcher thread passes new descriptors and
// releases, launches rounds (at most `max_rounds_in_flight` queued) while
// there is work, and reads the mailbox.  No kernel here waits on anything:
// the host sees an error of any launch through cudaStreamQuery and fails
// the server's outstanding requests.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/syev3.h"
#include "common.cuh"
#include "internal.h"

namespace {

using namespace syev3;

constexpr int kSlots = SYEV3_SERVER_SLOTS;  // request ring: outstanding requests
static_assert(kSlots <= kServeMaxItems && kServeMaxItems < (1 << 16), "item counts are 16-bit fields");
constexpr int kMaxNew = 48;                 // descriptors passed per round
constexpr int kMaxRel = 96;                 // releases passed per round
constexpr int kMailRing = 1 << 17;          // mailbox records: >= 2 per slot per round in flight
constexpr int64_t kUnit = 256;              // arena granule, bytes
constexpr int kCtlThreads = 256;

enum : int { kFree = 0, kQueued = 1, kAdmitted = 2, kDone = 3 };
enum : int { kListF64 = 0, kListF32 = 1, kListF32C = 2 };

// One request ring slot (device memory; written by the two control kernels).
struct DevReq {
  const void* A;
  int64_t n;
  uint64_t ticket;
  int32_t list;      // kListF64 / kListF32 / kListF32C
  int32_t vectors;
  int32_t state;
  int32_t pad;
  int64_t off;       // arena extent, in units
  int64_t units;
  int64_t lam_units; // eigenvalues first, eigenvectors from off + lam_units
  int64_t issued;    // matrices given to rounds
  int64_t finished;  // matrices solved
  uint64_t t_admit, t_done;  // %globaltimer
};

struct Extent {
  int64_t off, len;  // units
};

struct DevCtl {
  uint64_t head;      // tickets admitted (FIFO: the next is head + 1)
  uint64_t tail;      // tickets published by the host
  int64_t n_ext;      // free extents, sorted by offset, never adjacent
  int64_t used, peak; // arena units
  int64_t n_active;   // admitted requests with matrices not yet issued
  int64_t rr;         // round-robin position in `active`
  uint64_t n_rec;     // mailbox records published
  uint64_t rounds;
  uint64_t items;     // work items issued, all rounds
  int32_t active[kSlots];
  int64_t take[kSlots];  // the round's matrices per active position (scratch)
  Extent ext[kSlots + 1];
  ServeList lists[3];
};

// Mapped host memory, written by the device, read by the dispatcher.
struct MailRec {
  uint64_t ticket;
  int64_t off;      // arena units (admission)
  uint64_t t_dev;   // %globaltimer of the admission or completion
  int32_t kind;     // kAdmitted or kDone
  int32_t pad;
};

struct Mailbox {
  uint64_t n_rec;
  uint64_t rounds_done;
  uint64_t items;
  int64_t pending;  // matrices of admitted requests not yet issued (after the last admission)
  int64_t queued;   // requests waiting for memory
  int64_t used, peak;
  MailRec rec[kMailRing];
};

struct NewReq {
  const void* A;
  int64_t n;
  uint64_t ticket;
  int32_t list;
  int32_t vectors;
};

struct AdmitArgs {
  int32_t n_new, n_rel;
  int64_t chunk, round_matrices;
  NewReq nw[kMaxNew];
  int32_t rel[kMaxRel];
};
static_assert(sizeof(AdmitArgs) <= 4000, "kernel argument size");

__device__ __forceinline__ int64_t elem_bytes(int list) { return list == kListF64 ? 8 : 4; }

__device__ __forceinline__ void publish(DevCtl* ctl, Mailbox* mb, const MailRec& r) {
  volatile MailRec* dst = &mb->rec[ctl->n_rec % kMailRing];
  dst->ticket = r.ticket;
  dst->off = r.off;
  dst->t_dev = r.t_dev;
  dst->kind = r.kind;
  ctl->n_rec++;
}

// Thread 0 of the control CTA works the allocator; the CTA helps with the
// searches (warp 0 scans 32 extents per step) and with shifting the list.
// Every thread calls these with the same arguments (CTA-uniform control).

// Index of the first extent with len >= need, or -1.
__device__ int64_t find_fit(DevCtl* ctl, int64_t need, int64_t* s_k) {
  const int tid = threadIdx.x;
  if (tid == 0) *s_k = -1;
  __syncthreads();
  if (tid < 32) {
    const int64_t n = ctl->n_ext;
    for (int64_t b = 0; b < n; b += 32) {
      const int64_t i = b + tid;
      const bool fit = i < n && ctl->ext[i].len >= need;
      const unsigned m = __ballot_sync(0xffffffffu, fit);
      if (m) {
        if (tid == 0) *s_k = b + __ffs(m) - 1;
        break;
      }
    }
  }
  __syncthreads();
  return *s_k;
}

// Index of the first extent with off > x (n_ext if none).
__device__ int64_t find_after(DevCtl* ctl, int64_t x, int64_t* s_k) {
  const int tid = threadIdx.x;
  if (tid == 0) *s_k = ctl->n_ext;
  __syncthreads();
  if (tid < 32) {
    const int64_t n = ctl->n_ext;
    for (int64_t b = 0; b < n; b += 32) {
      const int64_t i = b + tid;
      const bool after = i < n && ctl->ext[i].off > x;
      const unsigned m = __ballot_sync(0xffffffffu, after);
      if (m) {
        if (tid == 0) *s_k = b + __ffs(m) - 1;
        break;
      }
    }
  }
  __syncthreads();
  return *s_k;
}

// Shift ext[k, n_ext) by `by` (+1: open a gap at k; -1: close the one at
// k - 1), in blocks that are read before they are written.
__device__ void shift_ext(DevCtl* ctl, int64_t k, int by) {
  const int64_t n = ctl->n_ext;
  const int tid = threadIdx.x;
  if (by > 0) {
    for (int64_t hi = n; hi > k; hi -= kCtlThreads) {
      const int64_t lo = hi - kCtlThreads > k ? hi - kCtlThreads : k;
      const int64_t i = lo + tid;
      Extent e{0, 0};
      if (i < hi) e = ctl->ext[i];
      __syncthreads();
      if (i < hi) ctl->ext[i + 1] = e;
      __syncthreads();
    }
  } else {
    for (int64_t lo = k; lo < n; lo += kCtlThreads) {
      const int64_t i = lo + tid;
      Extent e{0, 0};
      if (i < n) e = ctl->ext[i];
      __syncthreads();
      if (i < n) ctl->ext[i - 1] = e;
      __syncthreads();
    }
  }
  if (tid == 0) ctl->n_ext = n + by;
  __syncthreads();
}

// First-fit allocation of `need` units; -1 when no extent is large enough.
__device__ int64_t arena_alloc(DevCtl* ctl, int64_t need, int64_t* s_k) {
  const int64_t k = find_fit(ctl, need, s_k);
  if (k < 0) return -1;
  const Extent e = ctl->ext[k];
  __syncthreads();
  if (e.len == need) {
    shift_ext(ctl, k + 1, -1);
  } else if (threadIdx.x == 0) {
    ctl->ext[k].off = e.off + need;
    ctl->ext[k].len = e.len - need;
  }
  if (threadIdx.x == 0) {
    ctl->used += need;
    if (ctl->used > ctl->peak) ctl->peak = ctl->used;
  }
  __syncthreads();
  return e.off;
}

// Return [off, off + len) to the free list, merging with its neighbours.
__device__ void arena_free(DevCtl* ctl, int64_t off, int64_t len, int64_t* s_k) {
  const int64_t k = find_after(ctl, off, s_k);
  const bool prev = k > 0 && ctl->ext[k - 1].off + ctl->ext[k - 1].len == off;
  const bool next = k < ctl->n_ext && off + len == ctl->ext[k].off;
  __syncthreads();
  if (prev && next) {
    if (threadIdx.x == 0) ctl->ext[k - 1].len += len + ctl->ext[k].len;
    __syncthreads();
    shift_ext(ctl, k + 1, -1);
  } else if (prev) {
    if (threadIdx.x == 0) ctl->ext[k - 1].len += len;
  } else if (next) {
    if (threadIdx.x == 0) {
      ctl->ext[k].off = off;
      ctl->ext[k].len += len;
    }
  } else {
    shift_ext(ctl, k, +1);
    if (threadIdx.x == 0) ctl->ext[k] = Extent{off, len};
  }
  if (threadIdx.x == 0) ctl->used -= len;
  __syncthreads();
}

// Inclusive sum of v over the CTA's kCtlThreads threads (every thread calls
// it); *total receives the CTA's sum.
__device__ int64_t cta_inclusive_sum(int64_t v, int64_t* s_warp, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kCtlThreads / 32;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  const int64_t r = x + (warp > 0 ? s_warp[warp - 1] : 0);
  *total = s_warp[kWarps - 1];
  __syncthreads();  // s_warp is reused by the next call
  return r;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kCtlThreads) k_serve_admit(DevCtl* ctl, DevReq* reqs, Mailbox* mb, char* arena,
                                                              const AdmitArgs args) {
  __shared__ int64_t s_k;
  __shared__ int s_stop;
  __shared__ int64_t s_warp[kCtlThreads / 32];
  __shared__ int64_t s_first, s_rr;
  const int tid = threadIdx.x;
  // 1. Releases: the host passes only done requests it has not passed before.
  for (int r = 0; r < args.n_rel; ++r) {
    DevReq* q = &reqs[args.rel[r]];
    const int64_t off = q->off, len = q->units;
    __syncthreads();
    arena_free(ctl, off, len, &s_k);
    if (tid == 0) q->state = kFree;
  }
  // 2. New descriptors, in ticket order.
  if (tid < args.n_new) {
    const NewReq& nr = args.nw[tid];
    DevReq* q = &reqs[(nr.ticket - 1) % kSlots];
    const int64_t es = elem_bytes(nr.list);
    q->A = nr.A;
    q->n = nr.n;
    q->ticket = nr.ticket;
    q->list = nr.list;
    q->vectors = nr.vectors;
    q->state = kQueued;
    q->lam_units = (nr.n * 3 * es + kUnit - 1) / kUnit;
    q->units = q->lam_units + (nr.vectors ? (nr.n * 9 * es + kUnit - 1) / kUnit : 0);
    q->issued = 0;
    q->finished = 0;
    q->off = 0;
    q->t_admit = q->t_done = 0;
  }
  __syncthreads();
  if (tid == 0 && args.n_new > 0) ctl->tail = args.nw[args.n_new - 1].ticket;
  __syncthreads();
  // 3. Admission in arrival order while the arena has room.
  for (;;) {
    if (tid == 0) s_stop = (ctl->head >= ctl->tail);
    __syncthreads();
    if (s_stop) break;
    DevReq* q = &reqs[ctl->head % kSlots];  // ticket head + 1
    const int64_t need = q->units;
    __syncthreads();
    const int64_t off = arena_alloc(ctl, need, &s_k);
    if (off < 0) break;  // head of the line waits for memory
    if (tid == 0) {
      q->off = off;
      q->state = kAdmitted;
      q->t_admit = global_timer_ns();
      ctl->active[ctl->n_active++] = (int32_t)(ctl->head % kSlots);
      ctl->head++;
      publish(ctl, mb, MailRec{q->ticket, off, q->t_admit, kAdmitted, 0});
    }
    __syncthreads();
  }
  // 4. This round's work: round-robin over the admitted requests with
  // matrices left, at most `chunk` each and `round_matrices` in all, built
  // by the whole CTA with prefix sums over the active list taken in
  // round-robin order (position j is active[(start + j) % na]).
  const int64_t na = ctl->n_active;
  const int64_t start = na > 0 ? ctl->rr % na : 0;
  if (tid == 0) s_first = INT64_MAX;
  __syncthreads();
  // 4a. take_j = the part of min(chunk, left) within the round's budget.
  int64_t carry = 0;
  for (int64_t j0 = 0; j0 < na; j0 += kCtlThreads) {
    const int64_t j = j0 + tid;
    int64_t c = 0;
    if (j < na) {
      const DevReq* q = &reqs[ctl->active[(start + j) % na]];
      c = min(args.chunk, q->n - q->issued);
    }
    int64_t tot;
    const int64_t incl = cta_inclusive_sum(c, s_warp, &tot) + carry;
    if (j < na) {
      const int64_t t = min(max(args.round_matrices - (incl - c), (int64_t)0), c);
      ctl->take[j] = t;
      if (t < c) atomicMin(reinterpret_cast<unsigned long long*>(&s_first), (unsigned long long)j);
    }
    carry += tot;
  }
  __syncthreads();
  // 4b. Items: per list, an item index and a first tile from prefix sums of
  // packed counts (16 bits of items and 21 bits of tiles per list).
  uint64_t carry_i = 0, carry_t = 0;
  for (int64_t j0 = 0; j0 < na; j0 += kCtlThreads) {
    const int64_t j = j0 + tid;
    int64_t t = 0;
    int slot = 0, l = 0;
    if (j < na) {
      slot = ctl->active[(start + j) % na];
      t = ctl->take[j];
      l = reqs[slot].list;
    }
    const uint64_t tiles = (uint64_t)((t + kServeTile - 1) / kServeTile);
    const uint64_t vi = t > 0 ? (1ull << (16 * l)) : 0ull;
    const uint64_t vt = t > 0 ? (tiles << (21 * l)) : 0ull;
    int64_t ti, tt;
    const uint64_t ii = (uint64_t)cta_inclusive_sum((int64_t)vi, s_warp, &ti) + carry_i;
    const uint64_t it_ = (uint64_t)cta_inclusive_sum((int64_t)vt, s_warp, &tt) + carry_t;
    if (t > 0) {
      DevReq* q = &reqs[slot];
      ServeList* L = &ctl->lists[l];
      const int64_t idx = (int64_t)(((ii - vi) >> (16 * l)) & 0xffffull);
      const int64_t es = elem_bytes(l);
      char* out = arena + q->off * kUnit;
      ServeItem& item = L->items[idx];
      item.A = static_cast<const char*>(q->A) + q->issued * 6 * es;
      item.lam = out + q->issued * 3 * es;
      item.U = q->vectors ? out + q->lam_units * kUnit + q->issued * 9 * es : nullptr;
      item.count = t;
      item.tile_begin = (int64_t)(((it_ - vt) >> (21 * l)) & 0x1fffffull);
      item.tag = slot;
      q->issued += t;
    }
    carry_i += (uint64_t)ti;
    carry_t += (uint64_t)tt;
  }
  if (tid == 0) {
    int64_t items = 0;
    for (int l = 0; l < 3; ++l) {
      ctl->lists[l].n_items = (int64_t)((carry_i >> (16 * l)) & 0xffffull);
      ctl->lists[l].n_tiles = (int64_t)((carry_t >> (21 * l)) & 0x1fffffull);
      items += ctl->lists[l].n_items;
    }
    ctl->items += items;
  }
  __syncthreads();
  // 4c. Drop requests with nothing left to issue, keeping the order; the
  // next round starts at the first request this one did not serve in full.
  int64_t w0 = 0, pending = 0;
  if (tid == 0) s_rr = 0;
  for (int64_t a0 = 0; a0 < na; a0 += kCtlThreads) {
    const int64_t a = a0 + tid;
    int slot = -1;
    int64_t left = 0;
    if (a < na) {
      slot = ctl->active[a];
      left = reqs[slot].n - reqs[slot].issued;
    }
    const int64_t keep = left > 0 ? 1 : 0;
    int64_t kt, lt;
    const int64_t pos = cta_inclusive_sum(keep, s_warp, &kt) - keep + w0;
    cta_inclusive_sum(left, s_warp, &lt);
    if (keep) {
      ctl->active[pos] = slot;  // pos <= a: this block was read before the sums' barriers
      if (s_first != INT64_MAX && a == (start + s_first) % na) s_rr = pos;
    }
    w0 += kt;
    pending += lt;
    __syncthreads();
  }
  if (tid == 0) {
    ctl->n_active = w0;
    ctl->rr = w0 > 0 ? s_rr % w0 : 0;
    // Mirror the admission state (the records above first).
    __threadfence_system();
    volatile Mailbox* vm = mb;
    vm->pending = pending;
    vm->queued = (int64_t)(ctl->tail - ctl->head);
    vm->used = ctl->used;
    vm->peak = ctl->peak;
    vm->items = ctl->items;
    vm->n_rec = ctl->n_rec;
  }
}

__global__ void __launch_bounds__(kCtlThreads) k_serve_complete(DevCtl* ctl, DevReq* reqs, Mailbox* mb) {
  __shared__ int s_ndone;
  __shared__ uint64_t s_base;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_ndone = 0;
    s_base = ctl->n_rec;
  }
  __syncthreads();
  const uint64_t now = global_timer_ns();
  for (int l = 0; l < 3; ++l) {
    const ServeList* L = &ctl->lists[l];
    const int64_t ni = L->n_items;
    for (int64_t i = tid; i < ni; i += kCtlThreads) {  // one item per request per round
      const ServeItem& it = L->items[i];
      DevReq* q = &reqs[it.tag];
      q->finished += it.count;
      if (q->finished == q->n) {
        q->state = kDone;
        q->t_done = now;
        const int pos = atomicAdd(&s_ndone, 1);
        volatile MailRec* dst = &mb->rec[(s_base + pos) % kMailRing];
        dst->ticket = q->ticket;
        dst->off = q->off;
        dst->t_dev = now;
        dst->kind = kDone;
        __threadfence_system();  // the record before the count that publishes it
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    ctl->n_rec = s_base + s_ndone;
    ctl->rounds++;
    __threadfence_system();
    volatile Mailbox* vm = mb;
    vm->n_rec = ctl->n_rec;
    vm->rounds_done = ctl->rounds;
  }
}

__global__ void k_serve_init(DevCtl* ctl, int64_t arena_units) {
  ctl->head = ctl->tail = 0;
  ctl->n_ext = 1;
  ctl->ext[0] = Extent{0, arena_units};
  ctl->used = ctl->peak = 0;
  ctl->n_active = 0;
  ctl->rr = 0;
  ctl->n_rec = 0;
  ctl->rounds = 0;
  ctl->items = 0;
  for (int l = 0; l < 3; ++l) ctl->lists[l].n_items = ctl->lists[l].n_tiles = 0;
}

__global__ void k_read_timer(uint64_t* out) { *out = global_timer_ns(); }

using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

struct HostReq {
  uint64_t ticket;
  const void* A;
  int dtype;
  int list;
  int64_t n;
  bool vectors;
  int state = 0;  // syev3_request_info.state
  int64_t off = 0, lam_units = 0;
  int64_t t_submit = 0, t_admit = 0, t_done = 0;  // host steady clock
};

int list_of(int dtype) {
  return dtype == SYEV3_F64 ? kListF64 : (dtype == SYEV3_F32 ? kListF32 : kListF32C);
}

}  // namespace

struct syev3_server_s {
  syev3_server_config cfg{};
  int device = 0;
  int64_t arena_units = 0;
  char* arena = nullptr;
  DevCtl* ctl = nullptr;
  DevReq* dreqs = nullptr;
  Mailbox* mb = nullptr;      // host view of the mapped mailbox
  Mailbox* mb_dev = nullptr;  // its device address
  cudaStream_t stream = nullptr;
  int64_t clock_offset = 0;   // host steady ns - device %globaltimer ns

  std::mutex mu;
  std::condition_variable cv;
  std::unordered_map<uint64_t, HostReq> reqs;
  std::deque<uint64_t> new_q;  // submitted, not yet passed to the device
  std::deque<int> rel_q;       // released slots, not yet passed
  std::vector<char> slot_live;
  int64_t outstanding[3] = {0, 0, 0};  // not yet done, per list
  uint64_t next_ticket = 1;
  uint64_t rec_seen = 0;
  uint64_t rounds_launched = 0;
  int64_t launches = 0;
  int64_t completed = 0, matrices_done = 0, waiting = 0;
  int error = SYEV3_OK;
  int inject = SYEV3_OK;  // syev3_server_inject_failure: fail instead of the next launch
  bool stop = false;
  std::thread dispatcher;

  void run();
  void poll_mailbox();
  void fail_all(int status);
  bool launch_round(const AdmitArgs& a, const bool lists[3]);
};

void syev3_server_s::fail_all(int status) {
  if (error == SYEV3_OK) error = status;
  for (auto& kv : reqs)
    if (kv.second.state < 2) kv.second.state = 3;
  new_q.clear();
  cv.notify_all();
}

void syev3_server_s::poll_mailbox() {
  volatile Mailbox* vm = mb;
  const uint64_t n = vm->n_rec;
  std::atomic_thread_fence(std::memory_order_acquire);
  bool any = false;
  for (; rec_seen < n; ++rec_seen) {
    volatile MailRec* vr = &vm->rec[rec_seen % kMailRing];
    MailRec rc;
    rc.ticket = vr->ticket;
    rc.off = vr->off;
    rc.t_dev = vr->t_dev;
    rc.kind = vr->kind;
    const MailRec* r = &rc;
    auto it = reqs.find(r->ticket);
    if (it == reqs.end()) continue;
    HostReq& q = it->second;
    if (r->kind == kAdmitted && q.state == 0) {
      q.state = 1;
      q.off = r->off;
      q.t_admit = (int64_t)r->t_dev + clock_offset;
      waiting--;
      any = true;
    } else if (r->kind == kDone && q.state <= 1) {
      if (q.state == 0) {  // admitted and done in records of one poll
        q.off = r->off;
        waiting--;
      }
      q.state = 2;
      q.t_done = (int64_t)r->t_dev + clock_offset;
      if (q.t_admit == 0) q.t_admit = q.t_done;
      completed++;
      matrices_done += q.n;
      outstanding[q.list]--;
      any = true;
    }
  }
  if (any) cv.notify_all();
}

bool syev3_server_s::launch_round(const AdmitArgs& a, const bool lists[3]) {
  k_serve_admit<<<1, kCtlThreads, 0, stream>>>(ctl, dreqs, mb_dev, arena, a);
  cudaError_t e = cudaGetLastError();
  int n = 1;
  if (e == cudaSuccess && lists[kListF64]) {
    e = launch_f64_serve(&ctl->lists[kListF64], nullptr, stream);
    ++n;
  }
  if (e == cudaSuccess && lists[kListF32]) {
    e = launch_f32_serve(&ctl->lists[kListF32], false, nullptr, stream);
    ++n;
  }
  if (e == cudaSuccess && lists[kListF32C]) {
    e = launch_f32_serve(&ctl->lists[kListF32C], true, nullptr, stream);
    ++n;
  }
  if (e == cudaSuccess) {
    k_serve_complete<<<1, kCtlThreads, 0, stream>>>(ctl, dreqs, mb_dev);
    e = cudaGetLastError();
    ++n;
  }
  launches += n;
  if (e != cudaSuccess) {
    record_cuda_error(e);
    return false;
  }
  return true;
}

void syev3_server_s::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    poll_mailbox();
    const uint64_t done_rounds = static_cast<volatile Mailbox*>(mb)->rounds_done;
    const uint64_t inflight = rounds_launched - done_rounds;
    if (inflight > 0 && error == SYEV3_OK) {
      const cudaError_t e = cudaStreamQuery(stream);
      if (e != cudaSuccess && e != cudaErrorNotReady) {
        record_cuda_error(e);
        fail_all(SYEV3_ECUDA);
      }
    }
    if (stop && (inflight == 0 || error != SYEV3_OK)) break;
    const int64_t pending = static_cast<volatile Mailbox*>(mb)->pending;
    const bool want = error == SYEV3_OK && !stop &&
                      (!new_q.empty() || !rel_q.empty() || pending > 0);
    if (want && inflight < (uint64_t)cfg.max_rounds_in_flight) {
      AdmitArgs a;
      std::memset(&a, 0, sizeof(a));
      a.chunk = cfg.chunk;
      a.round_matrices = cfg.round_matrices;
      // Releases first, and new requests only in a round that passes every
      // release still queued: the device then frees a slot before a new
      // request that reuses it arrives (the host frees the slot at release).
      while (!rel_q.empty() && a.n_rel < kMaxRel) {
        a.rel[a.n_rel++] = rel_q.front();
        rel_q.pop_front();
      }
      while (rel_q.empty() && !new_q.empty() && a.n_new < kMaxNew) {
        const HostReq& q = reqs[new_q.front()];
        NewReq& d = a.nw[a.n_new++];
        d.A = q.A;
        d.n = q.n;
        d.ticket = q.ticket;
        d.list = q.list;
        d.vectors = q.vectors ? 1 : 0;
        new_q.pop_front();
      }
      bool lists[3];
      for (int l = 0; l < 3; ++l) lists[l] = outstanding[l] > 0;
      if (inject != SYEV3_OK) {  // a launch failure, made on the host
        fail_all(inject);
        continue;
      }
      ++rounds_launched;
      lk.unlock();
      const bool ok = launch_round(a, lists);
      lk.lock();
      if (!ok) fail_all(SYEV3_ECUDA);
      continue;
    }
    if (inflight > 0)
      cv.wait_for(lk, std::chrono::microseconds(20));
    else
      cv.wait_for(lk, std::chrono::milliseconds(20));
  }
}

namespace {

// Free what create allocated (any subset), in reverse order.
void free_server(syev3_server_s* s) {
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->mb) cudaFreeHost(s->mb);
  if (s->dreqs) cudaFree(s->dreqs);
  if (s->ctl) cudaFree(s->ctl);
  if (s->arena) cudaFree(s->arena);
  delete s;
}

}  // namespace

extern "C" {

int syev3_server_create(const syev3_server_config* cfg, syev3_server** out) {
  if (out == nullptr) return SYEV3_EINVAL;
  syev3_server_config c;
  c.memory_budget_bytes = (size_t)16 << 30;
  c.chunk = (int64_t)1 << 18;
  c.round_matrices = (int64_t)1 << 21;
  c.max_rounds_in_flight = 2;
  if (cfg) {
    if (cfg->memory_budget_bytes) c.memory_budget_bytes = cfg->memory_budget_bytes;
    if (cfg->chunk > 0) c.chunk = cfg->chunk;
    if (cfg->round_matrices > 0) c.round_matrices = cfg->round_matrices;
    if (cfg->max_rounds_in_flight > 0) c.max_rounds_in_flight = cfg->max_rounds_in_flight;
  }
  // At most 4 rounds queued: the mailbox ring then holds every record the
  // host has not read yet (2 x kSlots per round).
  // At most 2^27 matrices per round: the round's tiles per list are counted
  // in 21-bit fields by the admission kernel.
  if (c.memory_budget_bytes < (size_t)kUnit || c.chunk < 1 || c.round_matrices < 1 ||
      c.round_matrices > ((int64_t)1 << 27) || c.max_rounds_in_flight > 4)
    return SYEV3_EINVAL;
  auto* s = new syev3_server_s();
  s->cfg = c;
  s->arena_units = (int64_t)(c.memory_budget_bytes / kUnit);
  s->slot_live.assign(kSlots, 0);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->arena, (size_t)s->arena_units * kUnit);
  if (e == cudaSuccess) e = cudaMalloc(&s->ctl, sizeof(DevCtl));
  if (e == cudaSuccess) e = cudaMalloc(&s->dreqs, sizeof(DevReq) * kSlots);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->mb, sizeof(Mailbox), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->mb_dev, s->mb, 0);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    std::memset(s->mb, 0, sizeof(Mailbox));
    k_serve_init<<<1, 1, 0, s->stream>>>(s->ctl, s->arena_units);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(s->dreqs, 0, sizeof(DevReq) * kSlots, s->stream);
  if (e == cudaSuccess) {
    // The device timer against the host's steady clock: the midpoint of a
    // launch that reads it (the error is half the launch's round trip).
    uint64_t* t = &s->mb->items;  // scratch word of the mapped mailbox, reset below
    uint64_t* t_dev = &s->mb_dev->items;
    e = cudaStreamSynchronize(s->stream);
    const int64_t h0 = now_ns();
    if (e == cudaSuccess) {
      k_read_timer<<<1, 1, 0, s->stream>>>(t_dev);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    const int64_t h1 = now_ns();
    s->clock_offset = (h0 + h1) / 2 - (int64_t)*static_cast<volatile uint64_t*>(t);
    *t = 0;
  }
  if (e != cudaSuccess) {
    free_server(s);
    return record_cuda_error(e);
  }
  s->dispatcher = std::thread([s] { s->run(); });
  *out = s;
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
  cudaStreamSynchronize(srv->stream);
  cudaGetLastError();
  free_server(srv);
  return SYEV3_OK;
}

int syev3_server_submit(syev3_server* srv, int dtype, const void* d_A, int64_t n, int vectors, uint64_t* ticket) {
  if (srv == nullptr || ticket == nullptr || d_A == nullptr || n <= 0) return SYEV3_EINVAL;
  if (dtype != SYEV3_F64 && dtype != SYEV3_F32 && dtype != SYEV3_F32_COMPENSATED) return SYEV3_EINVAL;
  const int64_t es = dtype == SYEV3_F64 ? 8 : 4;
  if ((reinterpret_cast<uintptr_t>(d_A) % es) != 0) return SYEV3_EINVAL;
  const int64_t units = (n * 3 * es + kUnit - 1) / kUnit + (vectors ? (n * 9 * es + kUnit - 1) / kUnit : 0);
  if (units > srv->arena_units) return SYEV3_EINVAL;  // could never be admitted
  {
    std::lock_guard<std::mutex> g(srv->mu);
    if (srv->error != SYEV3_OK) return srv->error;
    if (srv->stop) return SYEV3_EINVAL;
    const int slot = (int)((srv->next_ticket - 1) % kSlots);
    if (srv->slot_live[slot]) return SYEV3_EAGAIN;  // the ring is full of unreleased requests
    srv->slot_live[slot] = 1;
    HostReq q;
    q.ticket = srv->next_ticket++;
    q.A = d_A;
    q.dtype = dtype;
    q.list = list_of(dtype);
    q.n = n;
    q.vectors = vectors != 0;
    q.lam_units = (n * 3 * es + kUnit - 1) / kUnit;
    q.t_submit = now_ns();
    *ticket = q.ticket;
    srv->outstanding[q.list]++;
    srv->waiting++;
    srv->new_q.push_back(q.ticket);
    srv->reqs.emplace(q.ticket, q);
  }
  srv->cv.notify_all();
  return SYEV3_OK;
}

int syev3_server_query(syev3_server* srv, uint64_t ticket, syev3_request_info* info) {
  if (srv == nullptr || info == nullptr) return SYEV3_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return SYEV3_EINVAL;
  const HostReq& r = it->second;
  const int64_t es = r.dtype == SYEV3_F64 ? 8 : 4;
  (void)es;
  info->state = r.state;
  info->n = r.n;
  info->dtype = r.dtype;
  const bool placed = r.state == 1 || r.state == 2;
  info->d_lambda = placed ? srv->arena + r.off * kUnit : nullptr;
  info->d_U = (placed && r.vectors) ? srv->arena + (r.off + r.lam_units) * kUnit : nullptr;
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
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return SYEV3_EINVAL;
    if (it->second.state >= 2) break;
    if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = srv->reqs.find(ticket);
      if (it == srv->reqs.end()) return SYEV3_EINVAL;
      if (it->second.state < 2) return SYEV3_ETIMEOUT;
    }
  }
  return it->second.state == 2 ? SYEV3_OK : srv->error;
}

int syev3_server_release(syev3_server* srv, uint64_t ticket) {
  if (srv == nullptr) return SYEV3_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end() || it->second.state < 2) return SYEV3_EINVAL;
    const int slot = (int)((ticket - 1) % kSlots);
    if (it->second.state == 2 && srv->error == SYEV3_OK) {
      srv->rel_q.push_back(slot);  // the device frees its memory in the next round
      srv->slot_live[slot] = 0;
    }
    // A failed request's slot and memory stay taken: after a failure the
    // device state is not trusted, and the server only accepts destroy.
    srv->reqs.erase(it);
  }
  srv->cv.notify_all();
  return SYEV3_OK;
}

int syev3_server_inject_failure(syev3_server* srv, int status) {
  if (srv == nullptr || status == SYEV3_OK) return SYEV3_EINVAL;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->inject = status;
  }
  srv->cv.notify_all();
  return SYEV3_OK;
}

int syev3_server_get_stats(syev3_server* srv, syev3_server_stats* st) {
  if (srv == nullptr || st == nullptr) return SYEV3_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  volatile Mailbox* vm = srv->mb;
  st->completed = srv->completed;
  st->matrices = srv->matrices_done;
  st->chunks = (int64_t)vm->items;
  st->waiting = srv->waiting;
  st->arena_bytes = (size_t)srv->arena_units * kUnit;
  st->arena_used = (size_t)vm->used * kUnit;
  st->arena_peak = (size_t)vm->peak * kUnit;
  st->error = srv->error;
  st->rounds = (int64_t)vm->rounds_done;
  st->launches = srv->launches;
  return SYEV3_OK;
}

}  // extern "C"
