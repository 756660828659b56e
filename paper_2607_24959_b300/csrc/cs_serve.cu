// cs_serve.cu -- serving: continuous batching of independent contact solves
// (each request: forward solve + IFT adjoint for its own g).
//
// A native scheduler thread owns the GPU side.  Requests are copied at
// submit and queued.  The device arena is split into `streams` slots, one
// CUDA stream each; whenever a slot is free the scheduler admits queued
// requests in arrival order while they fit the slot's bytes (admission by
// device memory) and up to max_batch of them, packs them into the slot's
// pinned staging buffer (instance table, claim orders, counters, inputs),
// issues one host-to-device copy, launches one fused kernel per (nv, m)
// bucket, copies the outputs back and records an event.  Completed slots are
// found by polling their events; their requests are marked done and the slot
// is reused.  Requests that arrive while other batches are on the GPU are
// admitted into the next free slot, so their work overlaps on the device.
// Nothing on the device ever waits for the host.
//
// Policy CS_SERVE_FIXED instead launches only full batches of fixed_batch
// requests (or what cs_serve_flush releases): the fixed-size-launch baseline.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "contact_solve.h"
#include "cs_host.h"
#include "cs_warp.cuh"

namespace cs {
namespace {

double now_s() {
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
  std::atomic<int> state{0};  // 0 queued, 1 on the GPU, 2 done
};

// Device bytes one request takes in a slot (inputs and outputs, aligned).
size_t request_bytes(int nv, int m) {
  const size_t f = 4;
  size_t in = al4((size_t)nv * nv) + al4((size_t)m * nv) + 2 * al4(nv) + 2 * al4(m) + al4(nv);
  size_t out = 2 * al4(nv) + al4(m) + al4((size_t)m * nv);
  return sizeof(cs_inst) + 4 /*order*/ + 8 /*status, iters*/ + f * (in + out);
}

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* d = nullptr;  // device region
  char* h = nullptr;  // pinned staging, same layout
  size_t cap = 0;
  bool busy = false;
  std::vector<std::shared_ptr<Req>> reqs;
  size_t out_off = 0, out_bytes = 0, out_floats = 0;  // output region within the slot
  size_t o_a = 0, o_dq = 0, o_dr = 0, o_dJ = 0, o_st = 0, o_it = 0;  // element offsets
  std::vector<cs_inst> inst;                   // the batch's instance table
  double t_launch = 0;
};

}  // namespace
}  // namespace cs

struct cs_server {
  cs_serve_config cfg{};
  int device = 0;
  char* d_arena = nullptr;
  std::vector<cs::Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<cs::Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<cs::Req>> tickets;
  cs::BufPool pool;  // request buffers, returned when a ticket is retired
  uint64_t next_ticket = 1;
  bool stop = false;
  bool flush = false;
  std::thread worker;
  // statistics
  std::atomic<long long> submitted{0}, completed{0}, batches{0}, batched_requests{0};
  std::atomic<int> inflight{0}, max_inflight{0};
  std::atomic<int> failed_launches{0};
};

namespace cs {
namespace {

// Pack the admitted requests into the slot and launch.  Called by the worker
// with the server lock released.  Returns false on a CUDA error (the requests
// are then completed with CS_ST_FAILED).
bool launch_slot(cs_server* S, Slot& sl) {
  const int n = (int)sl.reqs.size();
  // bucket the requests like an execution plan
  std::map<std::pair<int, int>, std::vector<int>> groups;
  std::map<std::pair<int, int>, std::pair<int, int>> maxima;
  for (int i = 0; i < n; ++i) {
    const auto& r = *sl.reqs[i];
    std::pair<int, int> key = uses_warp_kernel(r.nv, r.m)
                                  ? std::make_pair(nv_bucket(r.nv), mt_bucket(r.m))
                                  : std::make_pair(-((r.nv + 31) / 32), cta_rows_per_thread(r.m));
    groups[key].push_back(i);
    auto& mx = maxima[key];
    mx.first = std::max(mx.first, r.nv);
    mx.second = std::max(mx.second, r.m);
  }
  // layout (element offsets in floats from the slot base)
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
  const size_t fb = off;                       // float region start (bytes)
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
  cudaError_t err = cudaMemcpyAsync(sl.d, sl.h, in_bytes, cudaMemcpyHostToDevice, sl.stream);
  char* dF = sl.d + fb;
  float* dout = reinterpret_cast<float*>(sl.d + sl.out_off);
  csk::Params P;
  memset(&P, 0, sizeof(P));
  P.n = n;
  P.inst = reinterpret_cast<const cs_inst*>(sl.d + inst_off);
  P.M = reinterpret_cast<const float*>(dF) + oM;
  P.J = reinterpret_cast<const float*>(dF) + oJ;
  P.qfrc = reinterpret_cast<const float*>(dF) + oq;
  P.aref = reinterpret_cast<const float*>(dF) + oar;
  P.D = reinterpret_cast<const float*>(dF) + oD;
  P.g = reinterpret_cast<const float*>(dF) + og;
  P.total_M = (int64_t)tM;
  P.total_J = (int64_t)tJ;
  P.total_v = (int64_t)tv;
  P.total_r = (int64_t)tr;
  P.a = dout + sl.o_a;
  P.dqfrc = dout + sl.o_dq;
  P.daref = dout + sl.o_dr;
  P.dJ = dout + sl.o_dJ;
  P.status = reinterpret_cast<int32_t*>(dout + out_floats) + sl.o_st;
  P.iters = reinterpret_cast<int32_t*>(dout + out_floats) + sl.o_it;
  P.tol = S->cfg.tol;
  P.max_iter = S->cfg.max_iter;
  P.keep_factor = 1;
  int bi = 0, pos = 0;
  pos = 0;
  for (auto& kv : groups) {
    if (err != cudaSuccess) break;
    csk::Params Q = P;
    Q.n_work = (int)kv.second.size();
    Q.order = reinterpret_cast<const int32_t*>(sl.d + order_off) + pos;
    Q.counter = reinterpret_cast<int32_t*>(sl.d + ctr_off + 256 * bi);
    pos += Q.n_work;
    LaunchCfg lc;
    lc.warps_per_block = 2;
    const auto& mx = maxima[kv.first];
    if (kv.first.first < 0)
      err = launch_cta(csk::MODE_FUSED, mx.first, mx.second, Q, sl.stream, nullptr);
    else
      err = launch_warp(csk::MODE_FUSED, kv.first.first, 32 * kv.first.second, Q, lc, sl.stream,
                        nullptr);
    ++bi;
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(sl.h + sl.out_off, sl.d + sl.out_off, sl.out_bytes,
                          cudaMemcpyDeviceToHost, sl.stream);
  if (err == cudaSuccess) err = cudaEventRecord(sl.done, sl.stream);
  return err == cudaSuccess;
}

void finish_slot(cs_server* S, Slot& sl, bool ok) {
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
  S->completed += n;
  sl.reqs.clear();
  sl.busy = false;
  S->inflight--;
}

void worker_loop(cs_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progress = false;
    // completions
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      lk.unlock();
      finish_slot(S, sl, q == cudaSuccess);
      lk.lock();
      progress = true;
    }
    if (S->stop) {
      bool any = false;
      for (auto& sl : S->slots) any = any || sl.busy;
      if (!any) break;
    }
    // admissions
    for (auto& sl : S->slots) {
      if (sl.busy || S->queue.empty() || S->stop) continue;
      const bool fixed = S->cfg.policy == CS_SERVE_FIXED;
      if (fixed && (int)S->queue.size() < S->cfg.fixed_batch && !S->flush) break;
      size_t used = 0;
      const int limit = fixed ? S->cfg.fixed_batch : S->cfg.max_batch;
      // bytes for tables, counters and alignment slack
      const size_t slack = 256 * 24 + 1024;
      if (fixed) {
        while (!S->queue.empty() && (int)sl.reqs.size() < limit) {
          auto& r = S->queue.front();
          const size_t b = request_bytes(r->nv, r->m) + 64;
          if (used + b + slack > sl.cap && !sl.reqs.empty()) break;
          used += b;
          r->state.store(1, std::memory_order_relaxed);
          sl.reqs.push_back(r);
          S->queue.pop_front();
        }
      } else {
        // one kernel kind per batch (warp-sized or CTA-sized instances), in
        // arrival order within the kind, so small requests never wait for a
        // large one's kernel
        const bool kind = uses_warp_kernel(S->queue.front()->nv, S->queue.front()->m);
        for (auto it = S->queue.begin(); it != S->queue.end() && (int)sl.reqs.size() < limit;) {
          auto& r = *it;
          if (uses_warp_kernel(r->nv, r->m) != kind) {
            ++it;
            continue;
          }
          const size_t b = request_bytes(r->nv, r->m) + 64;
          if (used + b + slack > sl.cap && !sl.reqs.empty()) break;
          used += b;
          r->state.store(1, std::memory_order_relaxed);
          sl.reqs.push_back(r);
          it = S->queue.erase(it);
        }
      }
      if (S->queue.empty()) S->flush = false;
      if (sl.reqs.empty()) continue;
      sl.busy = true;
      const int inf = ++S->inflight;
      int mx = S->max_inflight.load();
      while (inf > mx && !S->max_inflight.compare_exchange_weak(mx, inf)) {
      }
      S->batches++;
      S->batched_requests += (long long)sl.reqs.size();
      const double t = now_s();
      for (auto& r : sl.reqs) r->t_start = t;
      lk.unlock();
      const bool ok = launch_slot(S, sl);
      if (!ok) {
        S->failed_launches++;
        cudaStreamSynchronize(sl.stream);
        finish_slot(S, sl, false);
      }
      lk.lock();
      progress = true;
    }
    if (!progress) S->cv.wait_for(lk, std::chrono::microseconds(20));
  }
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" {

int cs_serve_create(const cs_serve_config* cfg, cs_server** out) {
  if (!out) return set_error(CS_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (!cfg) return set_error(CS_EINVAL, "config must not be NULL");
  if (cfg->streams < 1 || cfg->streams > 16)
    return set_error(CS_EINVAL, "streams = %d outside 1..16", cfg->streams);
  if (cfg->arena_bytes < (size_t)cfg->streams * (1 << 20))
    return set_error(CS_EINVAL, "arena_bytes must be at least 1 MiB per stream");
  if (cfg->max_batch < 1) return set_error(CS_EINVAL, "max_batch must be >= 1");
  if (cfg->policy != CS_SERVE_CONTINUOUS && cfg->policy != CS_SERVE_FIXED)
    return set_error(CS_EINVAL, "unknown policy %d", cfg->policy);
  if (cfg->policy == CS_SERVE_FIXED && cfg->fixed_batch < 1)
    return set_error(CS_EINVAL, "fixed_batch must be >= 1");
  if (!(cfg->tol >= 0.f) || cfg->max_iter < 0)
    return set_error(CS_EINVAL, "tol must be >= 0 and max_iter >= 0");
  cs_server* S = new cs_server();
  S->cfg = *cfg;
  if (S->cfg.max_queue <= 0) S->cfg.max_queue = 1 << 20;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_arena, cfg->arena_bytes);
  if (e != cudaSuccess) {
    delete S;
    return set_error(CS_ENOMEM, "serve arena: %s", cudaGetErrorString(e));
  }
  const size_t per = (cfg->arena_bytes / cfg->streams) & ~(size_t)255;
  S->slots.resize(cfg->streams);
  for (int i = 0; i < cfg->streams && e == cudaSuccess; ++i) {
    Slot& sl = S->slots[i];
    sl.cap = per;
    sl.d = S->d_arena + (size_t)i * per;
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h, per, cudaHostAllocDefault);
  }
  if (e != cudaSuccess) {
    for (auto& sl : S->slots) {
      if (sl.h) cudaFreeHost(sl.h);
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.done) cudaEventDestroy(sl.done);
    }
    cudaFree(S->d_arena);
    delete S;
    return set_error(CS_ENOMEM, "serve slots: %s", cudaGetErrorString(e));
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return CS_OK;
}

int cs_serve_submit(cs_server* S, const cs_request* q, uint64_t* ticket) {
  if (!S || !q || !ticket) return set_error(CS_EINVAL, "server, request and ticket must not be NULL");
  if (q->nv < 1 || q->nv > 128 || q->m < 0 || q->m > 1024)
    return set_error(CS_EUNSUPPORTED, "request nv = %d, m = %d outside 1..128 x 0..1024", q->nv,
                     q->m);
  if (!uses_warp_kernel(q->nv, q->m) && cta_smem_bytes(q->nv, q->m) > device_smem_optin())
    return set_error(CS_EUNSUPPORTED, "request nv = %d, m = %d does not fit one CTA", q->nv, q->m);
  if (!q->M || !q->qfrc || !q->g || (q->m > 0 && (!q->J || !q->aref || !q->D)))
    return set_error(CS_EINVAL, "request data pointers must not be NULL");
  const size_t need = request_bytes(q->nv, q->m) + 256 * 24 + 2048;
  if (need > S->slots[0].cap)
    return set_error(CS_EUNSUPPORTED, "request needs %zu bytes, a slot has %zu", need,
                     S->slots[0].cap);
  auto r = std::make_shared<Req>();
  r->nv = q->nv;
  r->m = q->m;
  const size_t nn = (size_t)q->nv * q->nv, mn = (size_t)q->m * q->nv;
  r->in = S->pool.get(nn + mn + 2 * (size_t)q->nv + 2 * (size_t)q->m);
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
  r->out = S->pool.get(2 * (size_t)q->nv + q->m + mn);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->cfg.max_queue)
      return set_error(CS_EBUSY, "queue full (%d requests)", S->cfg.max_queue);
    r->ticket = S->next_ticket++;
    S->tickets[r->ticket] = r;
    S->queue.push_back(r);
  }
  S->submitted++;
  S->cv.notify_one();
  *ticket = r->ticket;
  return CS_OK;
}

namespace {
// Copy a finished request's outputs and times into res (outside the lock).
void fill_result(const Req* r, cs_result* res) {
  const float* o = r->out.data();
  if (res->a) memcpy(res->a, o, r->nv * 4);
  if (res->dqfrc) memcpy(res->dqfrc, o + r->nv, r->nv * 4);
  if (res->daref && r->m) memcpy(res->daref, o + 2 * r->nv, r->m * 4);
  if (res->dJ && r->m) memcpy(res->dJ, o + 2 * r->nv + r->m, (size_t)r->m * r->nv * 4);
  res->status = r->status;
  res->iters = r->iters;
  res->t_submit = r->t_submit;
  res->t_start = r->t_start;
  res->t_done = r->t_done;
}
}  // namespace

int cs_serve_poll(cs_server* S, uint64_t ticket, cs_result* res) {
  if (!S || !res) return set_error(CS_EINVAL, "server and result must not be NULL");
  std::shared_ptr<Req> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return set_error(CS_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
    r = it->second;
    if (r->state.load(std::memory_order_acquire) != 2) return CS_PENDING;
    S->tickets.erase(it);
  }
  fill_result(r.get(), res);
  S->pool.put(std::move(r->in));
  S->pool.put(std::move(r->out));
  return CS_OK;
}

int cs_serve_submit_batch(cs_server* S, int32_t n, const cs_request* reqs, uint64_t* tickets) {
  if (!S || (n > 0 && (!reqs || !tickets)) || n < 0)
    return set_error(CS_EINVAL, "server, requests and tickets must not be NULL");
  for (int32_t i = 0; i < n; ++i) {
    const int rc = cs_serve_submit(S, reqs + i, tickets + i);
    if (rc != CS_OK) return i > 0 ? i : rc;
  }
  return n;
}

int cs_serve_poll_batch(cs_server* S, int32_t n, const uint64_t* tickets, cs_result* res,
                        int32_t* done) {
  if (!S || n < 0 || (n > 0 && (!tickets || !res || !done)))
    return set_error(CS_EINVAL, "server, tickets, results and done must not be NULL");
  // one pass under the lock (a poller holding many tickets must not contend
  // with the scheduler once per ticket), outputs copied after it
  std::vector<std::pair<int32_t, std::shared_ptr<Req>>> ready;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (int32_t i = 0; i < n; ++i) {
      if (done[i] == 1) continue;  // collected by an earlier call
      auto it = S->tickets.find(tickets[i]);
      if (it == S->tickets.end()) {
        done[i] = -1;
        continue;
      }
      if (it->second->state.load(std::memory_order_acquire) != 2) {
        done[i] = 0;
        continue;
      }
      ready.emplace_back(i, it->second);
      S->tickets.erase(it);
    }
  }
  for (auto& pr : ready) {
    fill_result(pr.second.get(), res + pr.first);
    S->pool.put(std::move(pr.second->in));
    S->pool.put(std::move(pr.second->out));
    done[pr.first] = 1;
  }
  return (int)ready.size();
}

int cs_serve_cancel(cs_server* S, uint64_t ticket) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return set_error(CS_ENOTFOUND, "ticket %llu", (unsigned long long)ticket);
  if (it->second->state.load() != 0) return set_error(CS_EBUSY, "request already on the GPU");
  auto& q = S->queue;
  q.erase(std::remove(q.begin(), q.end(), it->second), q.end());
  S->tickets.erase(it);
  return CS_OK;
}

int cs_serve_flush(cs_server* S) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->flush = true;
  }
  S->cv.notify_one();
  return CS_OK;
}

int cs_serve_get_stats(cs_server* S, cs_serve_stats* st) {
  if (!S || !st) return set_error(CS_EINVAL, "server and stats must not be NULL");
  memset(st, 0, sizeof(*st));
  st->submitted = S->submitted.load();
  st->completed = S->completed.load();
  st->batches = S->batches.load();
  st->batched_requests = S->batched_requests.load();
  st->max_inflight = S->max_inflight.load();
  st->failed_launches = S->failed_launches.load();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    st->queued = (int64_t)S->queue.size();
  }
  return CS_OK;
}

void cs_serve_destroy(cs_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_one();
  if (S->worker.joinable()) S->worker.join();
  for (auto& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.h) cudaFreeHost(sl.h);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  if (S->d_arena) cudaFree(S->d_arena);
  delete S;
}

}  // extern "C"
