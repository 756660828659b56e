// cs_serve_core.h -- the serving scheduler, independent of the device API.
//
// Continuous batching of independent contact solves (each request: forward
// solve + IFT adjoint for its own g).  A native scheduler thread owns the
// device side.  Requests are copied at submit and queued.  The device arena
// is split into `streams` slots, one stream each; whenever a slot is free
// the scheduler admits queued requests in arrival order while they fit the
// slot's bytes (admission by device memory) and up to max_batch of them,
// packs them into the slot's pinned staging buffer (instance table, claim
// orders, counters, inputs), issues one host-to-device copy, launches one
// fused kernel per (nv, m) bucket, copies the outputs back and records an
// event.  Completed slots are found by polling their events; their requests
// are marked done and the slot is reused.  Requests that arrive while other
// batches are on the device are admitted into the next free slot, so their
// work overlaps.  Nothing on the device waits for the host.
//
// Policy CS_SERVE_FIXED instead launches only full batches of fixed_batch
// requests (or what cs_serve_flush releases): the fixed-size-launch baseline.
//
// Failures are handled on the host: a copy, launch or completion that fails
// completes that batch's requests with CS_ST_FAILED and frees the slot;
// later batches are unaffected.  A fault hook lets a caller make any of
// those steps fail on purpose (the device is not involved: the step is not
// issued).  Requests that wait in the queue longer than queue_timeout_ms
// are completed with CS_ST_TIMEOUT without being run.
//
// The device operations (memory, streams, events, copies, kernel launches)
// come from the Backend template parameter: the library instantiates it
// with the CUDA runtime (cs_serve.cu); the scheduler itself is plain C++.
#pragma once

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

#include "contact_solve.h"

namespace cs_serve {

inline double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

inline size_t al4(size_t n) { return (n + 3) & ~(size_t)3; }
inline size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

// Host buffer of a request (uninitialised floats; capacity a power of two).
struct Buf {
  std::unique_ptr<float[]> p;
  size_t cap = 0;
  float* data() { return p.get(); }
  const float* data() const { return p.get(); }
};

// Recycles request buffers by power-of-two size class: a fresh allocation per
// request (page faults on large mappings, zero-filling) made submission the
// bottleneck of a high-rate client.
struct BufPool {
  std::mutex mu;
  std::vector<Buf> free_[40];
  static int cls(size_t n) {
    int c = 0;
    while (((size_t)1 << c) < n) ++c;
    return c;
  }
  Buf get(size_t n) {
    const int c = cls(n ? n : 1);
    {
      std::lock_guard<std::mutex> lk(mu);
      if (!free_[c].empty()) {
        Buf b = std::move(free_[c].back());
        free_[c].pop_back();
        return b;
      }
    }
    Buf b;
    b.cap = (size_t)1 << c;
    b.p.reset(new float[b.cap]);
    return b;
  }
  void put(Buf&& b) {
    if (!b.p) return;
    const int c = cls(b.cap);
    std::lock_guard<std::mutex> lk(mu);
    if (free_[c].size() < 4096) free_[c].push_back(std::move(b));
  }
};

struct Req {
  uint64_t ticket = 0;
  int nv = 0, m = 0;
  Buf in;   // M, J, qfrc, aref, D, g (packed back to back)
  Buf out;  // a, dqfrc, daref, dJ
  int32_t status = 0, iters = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::atomic<int> state{0};  // 0 queued, 1 on the device, 2 done
};

// Device bytes one request takes in a slot (inputs and outputs, aligned).
inline size_t request_bytes(int nv, int m) {
  const size_t f = 4;
  size_t in = al4((size_t)nv * nv) + al4((size_t)m * nv) + 2 * al4(nv) + 2 * al4(m) + al4(nv);
  size_t out = 2 * al4(nv) + al4(m) + al4((size_t)m * nv);
  return sizeof(cs_inst) + 4 /*order*/ + 8 /*status, iters*/ + f * (in + out);
}

// Bytes of tables, counters and alignment slack a batch needs besides its
// requests' own.
constexpr size_t kBatchSlack = 256 * 24 + 1024;

// One bucket launch of a batch, described with plain addresses in the
// device's address space.
struct LaunchDesc {
  bool cta = false;        // one CTA per instance (else one warp)
  int nv_max = 0, m_max = 0;
  int n = 0, n_work = 0;
  const cs_inst* inst = nullptr;
  const float *M = nullptr, *J = nullptr, *qfrc = nullptr, *aref = nullptr, *D = nullptr,
              *g = nullptr;
  int64_t total_M = 0, total_J = 0, total_v = 0, total_r = 0;
  float *a = nullptr, *dqfrc = nullptr, *daref = nullptr, *dJ = nullptr;
  int32_t *status = nullptr, *iters = nullptr;
  const int32_t* order = nullptr;
  int32_t* counter = nullptr;
  float tol = 0.f;
  int32_t max_iter = 0;
};

// Auxiliary streams per slot: a batch's bucket kernels run side by side,
// the first on the slot's stream and the others on these, so that a batch
// waits for its slowest bucket rather than for the sum of them.
constexpr int kAuxStreams = 3;

struct Slot {
  void* stream = nullptr;
  void* done = nullptr;
  void* aux[kAuxStreams] = {};   // bucket streams besides `stream`
  void* fork = nullptr;          // recorded on `stream` after the upload
  void* join[kAuxStreams] = {};  // recorded on aux[a] after its kernels
  char* d = nullptr;  // device region
  char* h = nullptr;  // pinned staging, same layout
  size_t cap = 0;
  bool busy = false;
  int64_t seq = -1;   // batch number of the batch in flight
  std::vector<std::shared_ptr<Req>> reqs;
  size_t out_off = 0, out_bytes = 0, out_floats = 0;  // output region within the slot
  size_t o_a = 0, o_dq = 0, o_dr = 0, o_dJ = 0, o_st = 0, o_it = 0;  // element offsets
  std::vector<cs_inst> inst;                   // the batch's instance table
};

// The scheduler.  Backend provides (all host calls, 0 / true on success):
//   bool init();  void bind();                       (device of the server)
//   bool alloc_device(size_t, char**); void free_device(char*);
//   bool alloc_pinned(size_t, char**); void free_pinned(char*);
//   bool stream_create(void**); void stream_destroy(void*);
//   bool event_create(void**);  void event_destroy(void*);
//   bool h2d(void* dst, const void* src, size_t, void* stream);
//   bool d2h(void* dst, const void* src, size_t, void* stream);
//   bool launch(const LaunchDesc&, void* stream);
//   bool record(void* event, void* stream);
//   bool wait_event(void* stream, void* event);  // stream waits for event
//   int query(void* event);     // 0 done, 1 not yet, -1 failed
//   void sync(void* stream);
//   bool warp_sized(int nv, int m);          // one warp solves it (else a CTA)
//   std::pair<int, int> bucket(int nv, int m);   // kernel bucket of a request
//   bool fits(int nv, int m);                // some kernel takes it
//   int set_error(int code, const char* fmt, ...) (returns code)
template <class Backend>
struct Server {
  Backend be;
  cs_serve_config cfg{};
  char* d_arena = nullptr;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
  std::deque<uint64_t> done_list;  // tickets in completion order, not yet reported
  BufPool pool;  // request buffers, returned when a ticket is retired
  uint64_t next_ticket = 1;
  bool stop = false;
  bool flush = false;
  int64_t next_seq = 0;
  std::atomic<cs_serve_fault_fn> fault{nullptr};
  std::atomic<void*> fault_user{nullptr};
  std::thread worker;
  // statistics
  std::atomic<long long> submitted{0}, completed{0}, batches{0}, batched_requests{0},
      timed_out{0};
  std::atomic<int> inflight{0}, max_inflight{0};
  std::atomic<int> failed_launches{0};

  // ---------------------------------------------------------------- life
  int create(const cs_serve_config* c) {
    if (!c) return be.set_error(CS_EINVAL, "config must not be NULL");
    if (c->streams < 1 || c->streams > 16)
      return be.set_error(CS_EINVAL, "streams = %d outside 1..16", c->streams);
    if (c->arena_bytes < (size_t)c->streams * (1 << 20))
      return be.set_error(CS_EINVAL, "arena_bytes must be at least 1 MiB per stream");
    if (c->max_batch < 1) return be.set_error(CS_EINVAL, "max_batch must be >= 1");
    if (c->policy != CS_SERVE_CONTINUOUS && c->policy != CS_SERVE_FIXED)
      return be.set_error(CS_EINVAL, "unknown policy %d", c->policy);
    if (c->policy == CS_SERVE_FIXED && c->fixed_batch < 1)
      return be.set_error(CS_EINVAL, "fixed_batch must be >= 1");
    if (!(c->tol >= 0.f) || c->max_iter < 0)
      return be.set_error(CS_EINVAL, "tol must be >= 0 and max_iter >= 0");
    if (c->queue_timeout_ms < 0) return be.set_error(CS_EINVAL, "queue_timeout_ms must be >= 0");
    cfg = *c;
    if (cfg.max_queue <= 0) cfg.max_queue = 1 << 20;
    if (!be.init() || !be.alloc_device(c->arena_bytes, &d_arena))
      return be.set_error(CS_ENOMEM, "serve arena: device memory not available");
    const size_t per = (c->arena_bytes / c->streams) & ~(size_t)255;
    slots.resize(c->streams);
    bool ok = true;
    for (int i = 0; i < c->streams && ok; ++i) {
      Slot& sl = slots[i];
      sl.cap = per;
      sl.d = d_arena + (size_t)i * per;
      ok = be.stream_create(&sl.stream) && be.event_create(&sl.done) &&
           be.event_create(&sl.fork) && be.alloc_pinned(per, &sl.h);
      for (int a = 0; a < kAuxStreams && ok; ++a)
        ok = be.stream_create(&sl.aux[a]) && be.event_create(&sl.join[a]);
    }
    if (!ok) {
      release();
      return be.set_error(CS_ENOMEM, "serve slots: streams, events or pinned memory");
    }
    worker = std::thread([this] { worker_loop(); });
    return CS_OK;
  }

  void release() {
    for (auto& sl : slots) {
      if (sl.h) be.free_pinned(sl.h);
      if (sl.stream) be.stream_destroy(sl.stream);
      if (sl.done) be.event_destroy(sl.done);
      if (sl.fork) be.event_destroy(sl.fork);
      for (int a = 0; a < kAuxStreams; ++a) {
        if (sl.aux[a]) be.stream_destroy(sl.aux[a]);
        if (sl.join[a]) be.event_destroy(sl.join[a]);
        sl.aux[a] = sl.join[a] = nullptr;
      }
      sl.h = nullptr;
      sl.stream = sl.done = sl.fork = nullptr;
    }
    if (d_arena) be.free_device(d_arena);
    d_arena = nullptr;
  }

  void destroy() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_one();
    if (worker.joinable()) worker.join();
    for (auto& sl : slots) sync_slot(sl);
    release();
  }

  // Wait for everything a slot's batch issued, on all of its streams.
  void sync_slot(Slot& sl) {
    if (sl.stream) be.sync(sl.stream);
    for (int a = 0; a < kAuxStreams; ++a)
      if (sl.aux[a]) be.sync(sl.aux[a]);
  }

  // A fault hook step fails when the hook returns nonzero.
  bool injected(int stage, int64_t seq) {
    const cs_serve_fault_fn f = fault.load();
    return f && f(stage, seq, fault_user.load()) != 0;
  }

  // ---------------------------------------------------------- batches
  // Pack the admitted requests into the slot and launch.  Called by the
  // worker with the server lock released.  Returns false when a step failed
  // (the requests are then completed with CS_ST_FAILED).
  bool launch_slot(Slot& sl) {
    const int n = (int)sl.reqs.size();
    // bucket the requests like an execution plan
    std::map<std::pair<int, int>, std::vector<int>> groups;
    std::map<std::pair<int, int>, std::pair<int, int>> maxima;
    for (int i = 0; i < n; ++i) {
      const auto& r = *sl.reqs[i];
      const auto key = be.bucket(r.nv, r.m);
      groups[key].push_back(i);
      auto& mx = maxima[key];
      mx.first = std::max(mx.first, r.nv);
      mx.second = std::max(mx.second, r.m);
    }
    // layout (bytes from the slot base)
    size_t off = 0;
    const size_t inst_off = off;
    off += al256(n * sizeof(cs_inst));
    const size_t order_off = off;
    off += al256(n * sizeof(int32_t));
    const size_t ctr_off = off;
    off += 256 * groups.size();
    size_t tM = 0, tJ = 0, tv = 0, tr = 0;
    sl.inst.assign(n, cs_inst{});
    for (int i = 0; i < n; ++i) {
      const auto& r = *sl.reqs[i];
      cs_inst& e = sl.inst[i];
      e.nv = r.nv;
      e.m = r.m;
      e.off_M = (int64_t)tM;
      e.off_J = (int64_t)tJ;
      e.off_v = (int64_t)tv;
      e.off_r = (int64_t)tr;
      tM += al4((size_t)r.nv * r.nv);
      tJ += al4((size_t)r.m * r.nv);
      tv += al4(r.nv);
      tr += al4(r.m);
    }
    const size_t fb = off;  // float region start (bytes)
    const size_t oM = 0, oJ = oM + tM, oq = oJ + tJ, oar = oq + tv, oD = oar + tr, og = oD + tr;
    const size_t in_floats = og + tv;
    const size_t out_start = al256(fb + in_floats * 4);
    sl.o_a = 0;
    sl.o_dq = sl.o_a + tv;
    sl.o_dr = sl.o_dq + tv;
    sl.o_dJ = sl.o_dr + tr;
    const size_t out_floats = sl.o_dJ + tJ;
    sl.o_st = 0;
    sl.o_it = n;
    sl.out_off = out_start;
    sl.out_floats = out_floats;
    sl.out_bytes = out_floats * 4 + 8 * (size_t)n;
    if (sl.out_off + sl.out_bytes > sl.cap) return false;  // admission guarantees this
    // pack
    memcpy(sl.h + inst_off, sl.inst.data(), n * sizeof(cs_inst));
    int32_t* ord = reinterpret_cast<int32_t*>(sl.h + order_off);
    memset(sl.h + ctr_off, 0, 256 * groups.size());
    float* F = reinterpret_cast<float*>(sl.h + fb);
    for (int i = 0; i < n; ++i) {
      const auto& r = *sl.reqs[i];
      const cs_inst& e = sl.inst[i];
      const float* src = r.in.data();
      const size_t nn = (size_t)r.nv * r.nv, mn = (size_t)r.m * r.nv;
      memcpy(F + oM + e.off_M, src, nn * 4);
      src += nn;
      memcpy(F + oJ + e.off_J, src, mn * 4);
      src += mn;
      memcpy(F + oq + e.off_v, src, r.nv * 4);
      src += r.nv;
      memcpy(F + oar + e.off_r, src, r.m * 4);
      src += r.m;
      memcpy(F + oD + e.off_r, src, r.m * 4);
      src += r.m;
      memcpy(F + og + e.off_v, src, r.nv * 4);
    }
    // claim orders: per bucket, most expensive first
    {
      int opos = 0;
      for (auto& kv : groups) {
        auto& idx = kv.second;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
          const double nx = sl.reqs[x]->nv, mx = sl.reqs[x]->m;
          const double ny = sl.reqs[y]->nv, my = sl.reqs[y]->m;
          return mx * nx * nx + nx * nx * nx > my * ny * ny + ny * ny * ny;
        });
        for (size_t q = 0; q < idx.size(); ++q) ord[opos + q] = idx[q];
        opos += (int)idx.size();
      }
    }
    const size_t in_bytes = fb + in_floats * 4;
    if (injected(CS_SERVE_FAULT_H2D, sl.seq) || !be.h2d(sl.d, sl.h, in_bytes, sl.stream))
      return false;
    const float* dF = reinterpret_cast<const float*>(sl.d + fb);
    float* dout = reinterpret_cast<float*>(sl.d + sl.out_off);
    LaunchDesc L;
    L.n = n;
    L.inst = reinterpret_cast<const cs_inst*>(sl.d + inst_off);
    L.M = dF + oM;
    L.J = dF + oJ;
    L.qfrc = dF + oq;
    L.aref = dF + oar;
    L.D = dF + oD;
    L.g = dF + og;
    L.total_M = (int64_t)tM;
    L.total_J = (int64_t)tJ;
    L.total_v = (int64_t)tv;
    L.total_r = (int64_t)tr;
    L.a = dout + sl.o_a;
    L.dqfrc = dout + sl.o_dq;
    L.daref = dout + sl.o_dr;
    L.dJ = dout + sl.o_dJ;
    L.status = reinterpret_cast<int32_t*>(dout + out_floats) + sl.o_st;
    L.iters = reinterpret_cast<int32_t*>(dout + out_floats) + sl.o_it;
    L.tol = cfg.tol;
    L.max_iter = cfg.max_iter;
    // bucket 0 on the slot's stream, bucket b > 0 on aux[(b - 1) % kAux],
    // forked after the upload and joined before the download
    const int n_aux = std::min((int)groups.size() - 1, kAuxStreams);
    if (n_aux > 0) {
      if (!be.record(sl.fork, sl.stream)) return false;
      for (int a = 0; a < n_aux; ++a)
        if (!be.wait_event(sl.aux[a], sl.fork)) return false;
    }
    int bi = 0, pos = 0;
    for (auto& kv : groups) {
      LaunchDesc Q = L;
      Q.n_work = (int)kv.second.size();
      Q.order = reinterpret_cast<const int32_t*>(sl.d + order_off) + pos;
      Q.counter = reinterpret_cast<int32_t*>(sl.d + ctr_off + 256 * bi);
      Q.cta = !be.warp_sized(maxima[kv.first].first, maxima[kv.first].second);
      Q.nv_max = maxima[kv.first].first;
      Q.m_max = maxima[kv.first].second;
      pos += Q.n_work;
      void* s = bi == 0 ? sl.stream : sl.aux[(bi - 1) % kAuxStreams];
      if (injected(CS_SERVE_FAULT_LAUNCH, sl.seq) || !be.launch(Q, s)) return false;
      ++bi;
    }
    for (int a = 0; a < n_aux; ++a)
      if (!be.record(sl.join[a], sl.aux[a]) || !be.wait_event(sl.stream, sl.join[a]))
        return false;
    if (injected(CS_SERVE_FAULT_D2H, sl.seq) ||
        !be.d2h(sl.h + sl.out_off, sl.d + sl.out_off, sl.out_bytes, sl.stream))
      return false;
    return be.record(sl.done, sl.stream);
  }

  void finish_slot(Slot& sl, bool ok) {
    const double t = now_s();
    const int n = (int)sl.reqs.size();
    const float* out = reinterpret_cast<const float*>(sl.h + sl.out_off);
    // status and iters follow the float outputs
    const int32_t* st = reinterpret_cast<const int32_t*>(out + sl.out_floats);
    const int32_t* it = st + n;
    for (int i = 0; i < n; ++i) {
      auto& r = *sl.reqs[i];
      const cs_inst& e = sl.inst[i];
      if (ok) {
        float* o = r.out.data();
        memcpy(o, out + sl.o_a + e.off_v, r.nv * 4);
        memcpy(o + r.nv, out + sl.o_dq + e.off_v, r.nv * 4);
        memcpy(o + 2 * r.nv, out + sl.o_dr + e.off_r, r.m * 4);
        memcpy(o + 2 * r.nv + r.m, out + sl.o_dJ + e.off_J, (size_t)r.m * r.nv * 4);
        r.status = st[i];
        r.iters = it[i];
      } else {
        r.status = CS_ST_FAILED;
        r.iters = 0;
      }
      r.t_done = t;
      r.state.store(2, std::memory_order_release);
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto& r : sl.reqs) done_list.push_back(r->ticket);
    }
    completed += n;
    sl.reqs.clear();
    sl.busy = false;
    inflight--;
  }

  // Requests that have waited longer than queue_timeout_ms: completed with
  // CS_ST_TIMEOUT and dropped from the queue (caller holds the lock).
  bool expire_queued(double t) {
    if (cfg.queue_timeout_ms <= 0 || queue.empty()) return false;
    const double limit = 1e-3 * cfg.queue_timeout_ms;
    bool any = false;
    for (auto it = queue.begin(); it != queue.end();) {
      Req& r = **it;
      if (t - r.t_submit > limit) {
        r.status = CS_ST_TIMEOUT;
        r.iters = 0;
        r.t_start = r.t_done = t;
        r.state.store(2, std::memory_order_release);
        done_list.push_back(r.ticket);
        timed_out++;
        completed++;
        it = queue.erase(it);
        any = true;
      } else {
        ++it;
      }
    }
    if (queue.empty()) flush = false;
    return any;
  }

  void worker_loop() {
    be.bind();
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progress = false;
      // completions
      for (auto& sl : slots) {
        if (!sl.busy) continue;
        int q = be.query(sl.done);
        if (q == 1) continue;
        if (q == 0 && injected(CS_SERVE_FAULT_COMPLETE, sl.seq)) q = -1;
        lk.unlock();
        if (q != 0) {
          failed_launches++;
          sync_slot(sl);
        }
        finish_slot(sl, q == 0);
        lk.lock();
        progress = true;
      }
      if (stop) {
        bool any = false;
        for (auto& sl : slots) any = any || sl.busy;
        if (!any) break;
      }
      progress = expire_queued(now_s()) || progress;
      // admissions
      for (auto& sl : slots) {
        if (sl.busy || queue.empty() || stop) continue;
        const bool fixed = cfg.policy == CS_SERVE_FIXED;
        if (fixed && (int)queue.size() < cfg.fixed_batch && !flush) break;
        size_t used = 0;
        const int limit = fixed ? cfg.fixed_batch : cfg.max_batch;
        if (fixed) {
          while (!queue.empty() && (int)sl.reqs.size() < limit) {
            auto& r = queue.front();
            const size_t b = request_bytes(r->nv, r->m) + 64;
            if (used + b + kBatchSlack > sl.cap && !sl.reqs.empty()) break;
            used += b;
            r->state.store(1, std::memory_order_relaxed);
            sl.reqs.push_back(r);
            queue.pop_front();
          }
        } else {
          // one kernel kind per batch (warp-sized or CTA-sized instances), in
          // arrival order within the kind, so small requests never wait for
          // a large one's kernel
          const bool kind = be.warp_sized(queue.front()->nv, queue.front()->m);
          for (auto it = queue.begin(); it != queue.end() && (int)sl.reqs.size() < limit;) {
            auto& r = *it;
            if (be.warp_sized(r->nv, r->m) != kind) {
              ++it;
              continue;
            }
            const size_t b = request_bytes(r->nv, r->m) + 64;
            if (used + b + kBatchSlack > sl.cap && !sl.reqs.empty()) break;
            used += b;
            r->state.store(1, std::memory_order_relaxed);
            sl.reqs.push_back(r);
            it = queue.erase(it);
          }
        }
        if (queue.empty()) flush = false;
        if (sl.reqs.empty()) continue;
        sl.busy = true;
        sl.seq = next_seq++;
        const int inf = ++inflight;
        int mx = max_inflight.load();
        while (inf > mx && !max_inflight.compare_exchange_weak(mx, inf)) {
        }
        batches++;
        batched_requests += (long long)sl.reqs.size();
        const double t = now_s();
        for (auto& r : sl.reqs) r->t_start = t;
        lk.unlock();
        const bool ok = launch_slot(sl);
        if (!ok) {
          failed_launches++;
          sync_slot(sl);
          finish_slot(sl, false);
        }
        lk.lock();
        progress = true;
      }
      if (!progress) cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }

  // ------------------------------------------------------------ the API
  int submit(const cs_request* q, uint64_t* ticket) {
    if (!q || !ticket) return be.set_error(CS_EINVAL, "request and ticket must not be NULL");
    if (q->nv < 1 || q->nv > 128 || q->m < 0 || q->m > 1024)
      return be.set_error(CS_EUNSUPPORTED, "request nv = %d, m = %d outside 1..128 x 0..1024",
                          q->nv, q->m);
    if (!be.fits(q->nv, q->m))
      return be.set_error(CS_EUNSUPPORTED, "request nv = %d, m = %d does not fit one CTA", q->nv,
                          q->m);
    if (!q->M || !q->qfrc || !q->g || (q->m > 0 && (!q->J || !q->aref || !q->D)))
      return be.set_error(CS_EINVAL, "request data pointers must not be NULL");
    const size_t need = request_bytes(q->nv, q->m) + kBatchSlack + 1024;
    if (need > slots[0].cap)
      return be.set_error(CS_EUNSUPPORTED, "request needs %zu bytes, a slot has %zu", need,
                          slots[0].cap);
    auto r = std::make_shared<Req>();
    r->nv = q->nv;
    r->m = q->m;
    const size_t nn = (size_t)q->nv * q->nv, mn = (size_t)q->m * q->nv;
    r->in = pool.get(nn + mn + 2 * (size_t)q->nv + 2 * (size_t)q->m);
    float* d = r->in.data();
    memcpy(d, q->M, nn * 4);
    d += nn;
    if (mn) memcpy(d, q->J, mn * 4);
    d += mn;
    memcpy(d, q->qfrc, q->nv * 4);
    d += q->nv;
    if (q->m) memcpy(d, q->aref, q->m * 4);
    d += q->m;
    if (q->m) memcpy(d, q->D, q->m * 4);
    d += q->m;
    memcpy(d, q->g, q->nv * 4);
    r->out = pool.get(2 * (size_t)q->nv + q->m + mn);
    r->t_submit = now_s();
    {
      std::lock_guard<std::mutex> lk(mu);
      if ((int)queue.size() >= cfg.max_queue)
        return be.set_error(CS_EBUSY, "queue full (%d requests)", cfg.max_queue);
      r->ticket = next_ticket++;
      tickets[r->ticket] = r;
      queue.push_back(r);
    }
    submitted++;
    cv.notify_one();
    *ticket = r->ticket;
    return CS_OK;
  }

  // Copy a finished request's outputs and times into res (outside the lock).
  static void fill_result(const Req* r, cs_result* res) {
    const float* o = r->out.data();
    const bool have = r->status != CS_ST_FAILED && r->status != CS_ST_TIMEOUT;
    auto put = [&](float* dst, const float* src, size_t n) {
      if (!dst || !n) return;
      if (have) memcpy(dst, src, n * 4);
      else memset(dst, 0, n * 4);
    };
    put(res->a, o, r->nv);
    put(res->dqfrc, o + r->nv, r->nv);
    put(res->daref, o + 2 * r->nv, r->m);
    put(res->dJ, o + 2 * r->nv + r->m, (size_t)r->m * r->nv);
    res->status = r->status;
    res->iters = r->iters;
    res->t_submit = r->t_submit;
    res->t_start = r->t_start;
    res->t_done = r->t_done;
  }

  int poll(uint64_t ticket, cs_result* res) {
    if (!res) return be.set_error(CS_EINVAL, "result must not be NULL");
    std::shared_ptr<Req> r;
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = tickets.find(ticket);
      if (it == tickets.end())
        return be.set_error(CS_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
      r = it->second;
      if (r->state.load(std::memory_order_acquire) != 2) return CS_PENDING;
      tickets.erase(it);
    }
    fill_result(r.get(), res);
    pool.put(std::move(r->in));
    pool.put(std::move(r->out));
    return CS_OK;
  }

  int submit_batch(int32_t n, const cs_request* reqs, uint64_t* t) {
    if ((n > 0 && (!reqs || !t)) || n < 0)
      return be.set_error(CS_EINVAL, "requests and tickets must not be NULL");
    for (int32_t i = 0; i < n; ++i) {
      const int rc = submit(reqs + i, t + i);
      if (rc != CS_OK) return i > 0 ? i : rc;
    }
    return n;
  }

  // A load generator in the calling thread: reqs[i] is submitted once the
  // steady clock reaches t0 + t_arrival[i] (seconds, ascending), the ones
  // due together in one bulk call.  It sleeps while the next arrival is more
  // than 150 us away and yields closer to it; a full queue (CS_EBUSY) is
  // retried, any other failure ends the replay.  Returns the number queued
  // (n unless a submission failed), or the first failure's code if none was.
  int replay(int32_t n, const cs_request* reqs, const double* t_arrival, double t0,
             uint64_t* t) {
    if (n < 0 || (n > 0 && (!reqs || !t_arrival || !t)))
      return be.set_error(CS_EINVAL, "requests, arrival times and tickets must not be NULL");
    int32_t k = 0;
    while (k < n) {
      const double now = now_s();
      int32_t k1 = k;
      while (k1 < n && t0 + t_arrival[k1] <= now) ++k1;
      if (k1 > k) {
        const int got = submit_batch(k1 - k, reqs + k, t + k);
        if (got == CS_EBUSY) {
          std::this_thread::yield();
        } else if (got < 0) {
          return k > 0 ? k : got;
        } else {
          k += got;
        }
      } else {
        const double dt = t0 + t_arrival[k] - now;
        if (dt > 150e-6)
          std::this_thread::sleep_for(std::chrono::duration<double>(dt - 100e-6));
        else
          std::this_thread::yield();
      }
    }
    return k;
  }

  int poll_batch(int32_t n, const uint64_t* t, cs_result* res, int32_t* done) {
    if (n < 0 || (n > 0 && (!t || !res || !done)))
      return be.set_error(CS_EINVAL, "tickets, results and done must not be NULL");
    // one pass under the lock (a poller holding many tickets must not
    // contend with the scheduler once per ticket), outputs copied after it
    std::vector<std::pair<int32_t, std::shared_ptr<Req>>> ready;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (int32_t i = 0; i < n; ++i) {
        if (done[i] == 1) continue;  // collected by an earlier call
        auto it = tickets.find(t[i]);
        if (it == tickets.end()) {
          done[i] = -1;
          continue;
        }
        if (it->second->state.load(std::memory_order_acquire) != 2) {
          done[i] = 0;
          continue;
        }
        ready.emplace_back(i, it->second);
        tickets.erase(it);
      }
    }
    for (auto& pr : ready) {
      fill_result(pr.second.get(), res + pr.first);
      pool.put(std::move(pr.second->in));
      pool.put(std::move(pr.second->out));
      done[pr.first] = 1;
    }
    return (int)ready.size();
  }

  // Tickets completed since the last call, in completion order (at most max).
  int take_completed(int32_t max, uint64_t* out) {
    if (max < 0 || (max > 0 && !out)) return be.set_error(CS_EINVAL, "tickets must not be NULL");
    std::lock_guard<std::mutex> lk(mu);
    int n = 0;
    while (n < max && !done_list.empty()) {
      out[n++] = done_list.front();
      done_list.pop_front();
    }
    return n;
  }

  int cancel(uint64_t ticket) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = tickets.find(ticket);
    if (it == tickets.end())
      return be.set_error(CS_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
    if (it->second->state.load() != 0) return be.set_error(CS_EBUSY, "request no longer queued");
    auto& q = queue;
    q.erase(std::remove(q.begin(), q.end(), it->second), q.end());
    tickets.erase(it);
    return CS_OK;
  }

  int do_flush() {
    {
      std::lock_guard<std::mutex> lk(mu);
      flush = true;
    }
    cv.notify_one();
    return CS_OK;
  }

  int stats(cs_serve_stats* st) {
    if (!st) return be.set_error(CS_EINVAL, "stats must not be NULL");
    memset(st, 0, sizeof(*st));
    st->submitted = submitted.load();
    st->completed = completed.load();
    st->batches = batches.load();
    st->batched_requests = batched_requests.load();
    st->max_inflight = max_inflight.load();
    st->failed_launches = failed_launches.load();
    st->timed_out = timed_out.load();
    {
      std::lock_guard<std::mutex> lk(mu);
      st->queued = (int64_t)queue.size();
    }
    return CS_OK;
  }

  int set_fault_hook(cs_serve_fault_fn fn, void* user) {
    fault_user.store(user);
    fault.store(fn);
    return CS_OK;
  }
};

}  // namespace cs_serve
