// Test double of the serving scheduler's device (test infrastructure only):
// the scheduler of cs_serve_core.h instantiated on host memory, with
// "kernels" that do not solve anything -- they mark every instance solved
// (status OK, one step) and return a = qfrc, dqfrc = g and zero daref, dJ --
// and events that complete a set delay after they are recorded, so that
// several batches can be in flight.  It exercises the scheduler's queueing,
// admission, failure and timeout handling on a machine without a GPU.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <utility>

#include "contact_solve.h"
#include "cs_serve_core.h"

namespace {

thread_local char g_err[512];

struct FakeEvent {
  std::mutex mu;
  bool recorded = false;
  double ready_at = 0;
};

struct FakeBackend {
  int latency_us = 200;
  bool init() { return true; }
  void bind() {}
  bool alloc_device(size_t n, char** p) { return (*p = (char*)aligned_alloc(256, (n + 255) & ~(size_t)255)) != nullptr; }
  void free_device(char* p) { free(p); }
  bool alloc_pinned(size_t n, char** p) { return alloc_device(n, p); }
  void free_pinned(char* p) { free(p); }
  bool stream_create(void** s) { *s = new int(0); return true; }
  void stream_destroy(void* s) { delete (int*)s; }
  bool event_create(void** e) { *e = new FakeEvent(); return true; }
  void event_destroy(void* e) { delete (FakeEvent*)e; }
  bool h2d(void* d, const void* h, size_t n, void*) { memcpy(d, h, n); return true; }
  bool d2h(void* h, const void* d, size_t n, void*) { memcpy(h, d, n); return true; }
  bool launch(const cs_serve::LaunchDesc& L, void*) {
    for (int q = 0; q < L.n_work; ++q) {
      const int b = L.order[q];
      const cs_inst& e = L.inst[b];
      for (int j = 0; j < e.nv; ++j) {
        L.a[e.off_v + j] = L.qfrc[e.off_v + j];
        L.dqfrc[e.off_v + j] = L.g[e.off_v + j];
      }
      for (int i = 0; i < e.m; ++i) L.daref[e.off_r + i] = 0.f;
      for (int64_t k = 0; k < (int64_t)e.m * e.nv; ++k) L.dJ[e.off_J + k] = 0.f;
      L.status[b] = CS_ST_OK;
      L.iters[b] = 1;
    }
    return true;
  }
  bool record(void* ev, void*) {
    FakeEvent* e = (FakeEvent*)ev;
    std::lock_guard<std::mutex> lk(e->mu);
    e->recorded = true;
    e->ready_at = cs_serve::now_s() + 1e-6 * latency_us;
    return true;
  }
  // "kernels" run at launch, so a stream never has to wait for another
  bool wait_event(void*, void*) { return true; }
  int query(void* ev) {
    FakeEvent* e = (FakeEvent*)ev;
    std::lock_guard<std::mutex> lk(e->mu);
    return (!e->recorded || cs_serve::now_s() >= e->ready_at) ? 0 : 1;
  }
  void sync(void*) {}
  bool warp_sized(int nv, int m) { return nv <= 32 && m <= 256; }
  std::pair<int, int> bucket(int nv, int m) {
    return {nv <= 32 ? 32 : 128, m <= 256 ? 1 : 4};
  }
  bool fits(int, int) { return true; }
  int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
  }
};

using FakeServer = cs_serve::Server<FakeBackend>;

}  // namespace

extern "C" {

const char* fake_last_error(void) { return g_err; }

int fake_serve_create(const cs_serve_config* cfg, int latency_us, void** out) {
  FakeServer* S = new FakeServer();
  S->be.latency_us = latency_us;
  const int rc = S->create(cfg);
  if (rc != CS_OK) {
    delete S;
    *out = nullptr;
    return rc;
  }
  *out = S;
  return CS_OK;
}

int fake_serve_submit(void* S, const cs_request* q, uint64_t* t) {
  return ((FakeServer*)S)->submit(q, t);
}
int fake_serve_poll(void* S, uint64_t t, cs_result* r) { return ((FakeServer*)S)->poll(t, r); }
int fake_serve_flush(void* S) { return ((FakeServer*)S)->do_flush(); }
int fake_serve_get_stats(void* S, cs_serve_stats* st) { return ((FakeServer*)S)->stats(st); }
int fake_serve_set_fault_hook(void* S, cs_serve_fault_fn f, void* u) {
  return ((FakeServer*)S)->set_fault_hook(f, u);
}
int fake_serve_replay(void* S, int32_t n, const cs_request* reqs, const double* t_arrival,
                      double t0, uint64_t* t) {
  return ((FakeServer*)S)->replay(n, reqs, t_arrival, t0, t);
}
double fake_serve_clock(void) { return cs_serve::now_s(); }
void fake_serve_destroy(void* S) {
  ((FakeServer*)S)->destroy();
  delete (FakeServer*)S;
}

}  // extern "C"
