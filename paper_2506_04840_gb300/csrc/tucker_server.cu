// Serving loop: continuous batching of Tucker requests.
//
// A worker thread owns one CUDA stream and a device pool.  Each iteration it
//  1. admits queued requests in arrival order while their workspace fits in
//     the pool (first-fit over free ranges) and fewer than max_active are in
//     flight, zeroes their device state and compiles their programs;
//  2. builds one tick: the next phase of every admitted request, merged into
//     one launch per (position, step kind, tile class); uploads the tick's
//     job tables from a pinned ring slot and launches;
//  3. records the tick's event; a request whose last phase was in the tick
//     completes when that event has completed (its status word is copied to
//     pinned memory inside the tick), and its workspace returns to the pool.
// Up to kDepth ticks are in flight, so the host prepares tick t+1 while the
// GPU runs tick t, and requests that arrive meanwhile join the next tick.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "tk_program.h"

namespace tk {
namespace {

constexpr int kDepth = 3;                    // ticks in flight
constexpr int kRing = kDepth + 1;            // job-table slots
constexpr size_t kSlotBytes = 8u << 20;      // job tables per tick

// First-fit allocator over [0, cap) with coalescing of free ranges.
class RangePool {
 public:
  explicit RangePool(size_t cap) : cap_(cap) { free_[0] = cap; }
  bool take(size_t bytes, size_t* off) {
    bytes = al(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void give(size_t off, size_t bytes) {
    bytes = al(bytes);
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
  size_t capacity() const { return cap_; }

 private:
  size_t cap_;
  std::map<size_t, size_t> free_;
};

struct Request {
  uint64_t id = 0;
  tk_item item;
  double t_submit = 0, t_admit = 0;
  size_t off = 0, bytes = 0;
  int slot = -1;            // pinned status slot
  Problem prob;
  size_t pc = 0;            // next phase
};

struct Tick {
  cudaEvent_t ev;
  std::vector<std::unique_ptr<Request>> finishing;
};

}  // namespace

struct Server {
  int dev = 0;
  tk_shift rule = TK_SHIFT_PAPER;
  int max_active = 256;
  cudaStream_t st = nullptr;
  unsigned char* pool_base = nullptr;
  std::unique_ptr<RangePool> pool;
  int* pinned_status = nullptr;       // max_active slots
  std::vector<int> free_slots;
  unsigned char* host_ring = nullptr; // pinned, kRing slots
  unsigned char* dev_ring = nullptr;
  int ring_next = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<std::unique_ptr<Request>> pending;   // guarded by mu
  std::deque<tk_completion> done;                 // guarded by mu
  uint64_t next_id = 1, submitted = 0, completed = 0;  // guarded by mu
  bool stop = false;
  tk_status fatal = TK_OK;

  std::vector<std::unique_ptr<Request>> active;   // worker only
  std::deque<Tick> inflight;                      // worker only
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  cudaEvent_t get_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }

  void retire(Tick& t) {
    const double tn = now();
    std::vector<tk_completion> out;
    for (auto& r : t.finishing) {
      tk_completion c;
      c.id = r->id;
      c.status = pinned_status[r->slot];
      c.submit_s = r->t_submit;
      c.admit_s = r->t_admit;
      c.done_s = tn;
      out.push_back(c);
      pool->give(r->off, r->bytes);
      free_slots.push_back(r->slot);
    }
    ev_pool.push_back(t.ev);
    std::lock_guard<std::mutex> lk(mu);
    for (auto& c : out) done.push_back(c);
    completed += out.size();
    cv_done.notify_all();
  }

  // Retires finished ticks; with `block`, waits for the oldest one first.
  void reap(bool block) {
    while (!inflight.empty()) {
      Tick& t = inflight.front();
      cudaError_t q = block ? cudaEventSynchronize(t.ev) : cudaEventQuery(t.ev);
      if (q == cudaErrorNotReady) return;
      if (q != cudaSuccess) fatal = TK_ECUDA;
      retire(t);
      inflight.pop_front();
      block = false;
    }
  }

  void admit() {
    std::lock_guard<std::mutex> lk(mu);
    while (!pending.empty() && (int)active.size() < max_active && !free_slots.empty()) {
      Request* r = pending.front().get();
      size_t off = 0;
      if (!pool->take(r->prob.ws_bytes, &off)) break;   // wait for memory (arrival order)
      std::unique_ptr<Request> rq = std::move(pending.front());
      pending.pop_front();
      rq->off = off;
      rq->bytes = rq->prob.ws_bytes;
      rq->slot = free_slots.back();
      free_slots.pop_back();
      rq->t_admit = now();
      problem_build(rq->item, pool_base + off, &rq->prob);
      cudaMemsetAsync(rq->prob.state, 0, sizeof(ItemState), st);
      active.push_back(std::move(rq));
    }
  }

  void tick() {
    std::vector<const Op*> ops;
    for (auto& r : active)
      for (const Op& o : r->prob.prog[r->pc]) ops.push_back(&o);
    std::vector<unsigned char> blob;
    std::vector<LaunchRec> recs;
    merge_ops(ops, blob, recs);
    if (blob.size() > kSlotBytes) {   // cannot happen below max_active = 4096
      fatal = TK_ENOTIMPL;
      return;
    }
    const int slot = ring_next;
    ring_next = (ring_next + 1) % kRing;
    unsigned char* hs = host_ring + (size_t)slot * kSlotBytes;
    unsigned char* ds = dev_ring + (size_t)slot * kSlotBytes;
    std::memcpy(hs, blob.data(), blob.size());
    cudaMemcpyAsync(ds, hs, blob.size(), cudaMemcpyHostToDevice, st);
    resolve(recs, ds);
    for (const auto& rc : recs)
      if (issue(rc, st, false) != cudaSuccess) fatal = TK_ECUDA;
    Tick t;
    std::vector<std::unique_ptr<Request>> still;
    for (auto& r : active) {
      r->pc++;
      if (r->pc == r->prob.prog.size()) {
        cudaMemcpyAsync(&pinned_status[r->slot], &r->prob.state->status, sizeof(int),
                        cudaMemcpyDeviceToHost, st);
        t.finishing.push_back(std::move(r));
      } else {
        still.push_back(std::move(r));
      }
    }
    active.swap(still);
    t.ev = get_event();
    cudaEventRecord(t.ev, st);
    inflight.push_back(std::move(t));
  }

  void run() {
    cudaSetDevice(dev);
    for (;;) {
      reap(false);
      admit();
      if (active.empty()) {
        if (!inflight.empty()) {
          reap(true);
          continue;
        }
        std::unique_lock<std::mutex> lk(mu);
        if (stop && pending.empty()) break;
        cv.wait_for(lk, std::chrono::milliseconds(1));
        continue;
      }
      if ((int)inflight.size() >= kDepth) reap(true);
      tick();
    }
  }
};

}  // namespace tk

using namespace tk;

extern "C" {

struct tk_server_s {
  Server* s;
};

tk_status tucker_server_create(const tk_server_opts* o, tk_server* out) {
  if (!o || !out) return TK_EINVAL;
  *out = nullptr;
  if (o->rule != TK_SHIFT_PAPER && o->rule != TK_SHIFT_NONE) return TK_EINVAL;
  if (o->max_active < 0 || o->max_active > 4096) return TK_EINVAL;
  auto* s = new Server;
  cudaGetDevice(&s->dev);
  s->rule = o->rule;
  s->max_active = o->max_active ? o->max_active : 256;
  size_t bytes = o->pool_bytes;
  if (bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    bytes = fr / 2;
  }
  bytes = al(bytes);
  tk_status st = TK_OK;
  if (cudaMalloc((void**)&s->pool_base, bytes) != cudaSuccess) st = TK_ENOMEM;
  if (st == TK_OK && cudaMallocHost((void**)&s->pinned_status, sizeof(int) * s->max_active) !=
                         cudaSuccess)
    st = TK_ENOMEM;
  if (st == TK_OK && cudaMallocHost((void**)&s->host_ring, kSlotBytes * kRing) != cudaSuccess)
    st = TK_ENOMEM;
  if (st == TK_OK && cudaMalloc((void**)&s->dev_ring, kSlotBytes * kRing) != cudaSuccess)
    st = TK_ENOMEM;
  if (st == TK_OK && cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess)
    st = TK_ECUDA;
  if (st != TK_OK) {
    if (s->pool_base) cudaFree(s->pool_base);
    if (s->pinned_status) cudaFreeHost(s->pinned_status);
    if (s->host_ring) cudaFreeHost(s->host_ring);
    if (s->dev_ring) cudaFree(s->dev_ring);
    cudaGetLastError();
    delete s;
    return st;
  }
  batch_kernels_init();
  s->pool.reset(new RangePool(bytes));
  for (int i = s->max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread([s] { s->run(); });
  *out = new tk_server_s{s};
  return TK_OK;
}

tk_status tucker_server_submit(tk_server h, const tk_item* item, uint64_t* id) {
  if (!h || !h->s || !item) return TK_EINVAL;
  Server* s = h->s;
  std::unique_ptr<Request> r(new Request);
  r->item = *item;
  tk_status st = problem_plan(r->item, s->rule, &r->prob);
  if (st != TK_OK) return st;
  if (al(r->prob.ws_bytes) > s->pool->capacity()) return TK_ENOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return TK_EINVAL;
  r->id = s->next_id++;
  r->t_submit = s->now();
  if (id) *id = r->id;
  s->pending.push_back(std::move(r));
  s->submitted++;
  s->cv.notify_all();
  return TK_OK;
}

int tucker_server_poll(tk_server h, tk_completion* out, int max) {
  if (!h || !h->s || !out || max <= 0) return 0;
  Server* s = h->s;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

tk_status tucker_server_drain(tk_server h, double timeout_s) {
  if (!h || !h->s) return TK_EINVAL;
  Server* s = h->s;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(
      lk, std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s),
      [s] { return s->completed == s->submitted; });
  if (s->fatal != TK_OK) return s->fatal;
  return ok ? TK_OK : TK_ETIMEOUT;
}

double tucker_server_clock(tk_server h) {
  if (!h || !h->s) return 0.0;
  return h->s->now();
}

tk_status tucker_server_destroy(tk_server h) {
  if (!h || !h->s) return TK_EINVAL;
  Server* s = h->s;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->worker.join();
  cudaStreamSynchronize(s->st);
  for (auto e : s->ev_pool) cudaEventDestroy(e);
  cudaStreamDestroy(s->st);
  cudaFree(s->pool_base);
  cudaFree(s->dev_ring);
  cudaFreeHost(s->pinned_status);
  cudaFreeHost(s->host_ring);
  const tk_status f = s->fatal;
  delete s;
  delete h;
  return f;
}

}  // extern "C"
