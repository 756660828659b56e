// cs_serve.cu -- serving: the scheduler of cs_serve_core.h on the CUDA
// runtime, and the C ABI's cs_serve_* entry points.
//
// The backend below maps the scheduler's device operations to the runtime
// (device arena, pinned staging, one stream and event per slot, async copies)
// and a batch's bucket launches to the fused kernels (one warp or one CTA
// per instance, claims in the order the scheduler packed).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <utility>

#include "contact_solve.h"
#include "cs_host.h"
#include "cs_serve_core.h"
#include "cs_warp.cuh"

namespace cs {
namespace {

struct CudaBackend {
  int device = 0;
  bool init() { return cudaGetDevice(&device) == cudaSuccess; }
  void bind() { cudaSetDevice(device); }
  bool alloc_device(size_t n, char** p) {
    return cudaMalloc(reinterpret_cast<void**>(p), n) == cudaSuccess;
  }
  void free_device(char* p) { cudaFree(p); }
  bool alloc_pinned(size_t n, char** p) {
    return cudaHostAlloc(reinterpret_cast<void**>(p), n, cudaHostAllocDefault) == cudaSuccess;
  }
  void free_pinned(char* p) { cudaFreeHost(p); }
  bool stream_create(void** s) {
    return cudaStreamCreateWithFlags(reinterpret_cast<cudaStream_t*>(s),
                                     cudaStreamNonBlocking) == cudaSuccess;
  }
  void stream_destroy(void* s) { cudaStreamDestroy((cudaStream_t)s); }
  bool event_create(void** e) {
    return cudaEventCreateWithFlags(reinterpret_cast<cudaEvent_t*>(e),
                                    cudaEventDisableTiming) == cudaSuccess;
  }
  void event_destroy(void* e) { cudaEventDestroy((cudaEvent_t)e); }
  bool h2d(void* d, const void* h, size_t n, void* s) {
    return cudaMemcpyAsync(d, h, n, cudaMemcpyHostToDevice, (cudaStream_t)s) == cudaSuccess;
  }
  bool d2h(void* h, const void* d, size_t n, void* s) {
    return cudaMemcpyAsync(h, d, n, cudaMemcpyDeviceToHost, (cudaStream_t)s) == cudaSuccess;
  }
  bool launch(const cs_serve::LaunchDesc& L, void* s) {
    csk::Params P;
    memset(&P, 0, sizeof(P));
    P.n = L.n;
    P.n_work = L.n_work;
    P.inst = L.inst;
    P.M = L.M;
    P.J = L.J;
    P.qfrc = L.qfrc;
    P.aref = L.aref;
    P.D = L.D;
    P.g = L.g;
    P.total_M = L.total_M;
    P.total_J = L.total_J;
    P.total_v = L.total_v;
    P.total_r = L.total_r;
    P.a = L.a;
    P.dqfrc = L.dqfrc;
    P.daref = L.daref;
    P.dJ = L.dJ;
    P.status = L.status;
    P.iters = L.iters;
    P.order = L.order;
    P.counter = L.counter;
    P.tol = L.tol;
    P.max_iter = L.max_iter;
    P.keep_factor = 1;
    cudaError_t e;
    if (L.cta) {
      e = launch_cta(csk::MODE_FUSED, L.nv_max, L.m_max, P, (cudaStream_t)s, nullptr);
    } else {
      LaunchCfg lc;
      lc.warps_per_block = 2;
      e = launch_warp(csk::MODE_FUSED, L.nv_max, L.m_max, P, lc, (cudaStream_t)s, nullptr);
    }
    return e == cudaSuccess;
  }
  bool record(void* ev, void* s) {
    return cudaEventRecord((cudaEvent_t)ev, (cudaStream_t)s) == cudaSuccess;
  }
  bool wait_event(void* s, void* ev) {
    return cudaStreamWaitEvent((cudaStream_t)s, (cudaEvent_t)ev, 0) == cudaSuccess;
  }
  int query(void* ev) {
    const cudaError_t q = cudaEventQuery((cudaEvent_t)ev);
    return q == cudaSuccess ? 0 : q == cudaErrorNotReady ? 1 : -1;
  }
  void sync(void* s) { cudaStreamSynchronize((cudaStream_t)s); }
  bool warp_sized(int nv, int m) { return uses_warp_kernel(nv, m); }
  std::pair<int, int> bucket(int nv, int m) {
    return uses_warp_kernel(nv, m) ? std::make_pair(nv_bucket(nv), mt_bucket(m))
                                   : std::make_pair(-((nv + 31) / 32), cta_rows_per_thread(m));
  }
  bool fits(int nv, int m) {
    return uses_warp_kernel(nv, m) || cta_smem_bytes(nv, m) <= device_smem_optin();
  }
  int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return cs::set_error(code, "%s", buf);
  }
};

}  // namespace
}  // namespace cs

struct cs_server : cs_serve::Server<cs::CudaBackend> {};

using namespace cs;

extern "C" {

int cs_serve_create(const cs_serve_config* cfg, cs_server** out) {
  if (!out) return set_error(CS_EINVAL, "out must not be NULL");
  *out = nullptr;
  cs_server* S = new cs_server();
  const int rc = S->create(cfg);
  if (rc != CS_OK) {
    delete S;
    return rc;
  }
  *out = S;
  return CS_OK;
}

int cs_serve_submit(cs_server* S, const cs_request* q, uint64_t* ticket) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->submit(q, ticket);
}

int cs_serve_poll(cs_server* S, uint64_t ticket, cs_result* res) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->poll(ticket, res);
}

int cs_serve_submit_batch(cs_server* S, int32_t n, const cs_request* reqs, uint64_t* tickets) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->submit_batch(n, reqs, tickets);
}

int cs_serve_replay(cs_server* S, int32_t n, const cs_request* reqs, const double* t_arrival,
                    double t0, uint64_t* tickets) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->replay(n, reqs, t_arrival, t0, tickets);
}

double cs_serve_clock(void) { return cs_serve::now_s(); }

int cs_serve_poll_batch(cs_server* S, int32_t n, const uint64_t* tickets, cs_result* res,
                        int32_t* done) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->poll_batch(n, tickets, res, done);
}

int cs_serve_completed(cs_server* S, int32_t max, uint64_t* tickets) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->take_completed(max, tickets);
}

int cs_serve_cancel(cs_server* S, uint64_t ticket) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->cancel(ticket);
}

int cs_serve_flush(cs_server* S) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->do_flush();
}

int cs_serve_get_stats(cs_server* S, cs_serve_stats* st) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->stats(st);
}

int cs_serve_set_fault_hook(cs_server* S, cs_serve_fault_fn hook, void* user) {
  if (!S) return set_error(CS_EINVAL, "server must not be NULL");
  return S->set_fault_hook(hook, user);
}

void cs_serve_destroy(cs_server* S) {
  if (!S) return;
  S->destroy();
  delete S;
}

}  // extern "C"
