// cs_api.cu -- host side of the C ABI declared in include/contact_solve.h:
// argument validation, kernel selection over the compiled (NV, MT) grid,
// launch geometry, and error reporting.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>

#include "contact_solve.h"
#include "cs_host.h"
#include "cs_warp.cuh"

namespace cs {

static thread_local char g_last_error[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* where) {
  return set_error(CS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Compiled buckets.  nv is padded up to the bucket; m up to 32 * MT.
static const int kNvBuckets[] = {3, 9, 18, 32};
static const int kMtBuckets[] = {1, 2, 3, 4, 6, 8};

int nv_bucket(int nv) {
  for (int b : kNvBuckets)
    if (nv <= b) return b;
  return -1;
}
int mt_bucket(int m) {
  for (int t : kMtBuckets)
    if (m <= 32 * t) return t;
  return -1;
}

struct DevInfo {
  int sms = 0;
  size_t smem_optin = 0;
};
static DevInfo dev_info() {
  static std::mutex mu;
  static DevInfo cache[16];
  static bool have[16] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return DevInfo{148, 227 * 1024};
  std::lock_guard<std::mutex> lk(mu);
  if (!have[dev]) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
      cache[dev].sms = p.multiProcessorCount;
      cache[dev].smem_optin = p.sharedMemPerBlockOptin;
    } else {
      cache[dev].sms = 148;
      cache[dev].smem_optin = 227 * 1024;
    }
    have[dev] = true;
  }
  return cache[dev];
}

int device_sm_count() { return dev_info().sms; }
size_t device_smem_optin() { return dev_info().smem_optin; }

cudaError_t launch_warp(int mode, int nv_max, int m_max, const csk::Params& P,
                        const LaunchCfg& cfg, cudaStream_t s, KernelInfo* info) {
  int nvb = nv_bucket(nv_max), mt = mt_bucket(m_max);
  if (nvb < 0 || mt < 0) return cudaErrorInvalidValue;
  switch (nvb) {
    case 3: return launch_nv<3>(mode, mt, P, cfg, s, info);
    case 9: return launch_nv<9>(mode, mt, P, cfg, s, info);
    case 18: return launch_nv<18>(mode, mt, P, cfg, s, info);
    default: return launch_nv<32>(mode, mt, P, cfg, s, info);
  }
}

bool uses_warp_kernel(int nv_max, int m_max) { return nv_max <= 32 && m_max <= 256; }

cudaError_t launch_dispatch(int mode, int nv_max, int m_max, const csk::Params& P,
                            const LaunchCfg& cfg, cudaStream_t s, KernelInfo* info) {
  if (uses_warp_kernel(nv_max, m_max)) return launch_warp(mode, nv_max, m_max, P, cfg, s, info);
  return launch_cta(mode, nv_max, m_max, P, s, info);
}

int launch_error(cudaError_t e, const char* where) {
  if (e == cudaErrorInvalidConfiguration)
    return set_error(CS_EUNSUPPORTED, "%s: the instance sizes do not fit one CTA's shared memory",
                     where);
  return cuda_error(e, where);
}

int check_batch(const cs_batch* b, const cs_options* o) {
  int rc = check_batch_shapes(b, o);
  if (rc != CS_OK || b->n == 0) return rc;
  if (!uses_warp_kernel(b->nv_max, b->m_max) &&
      cta_smem_bytes(b->nv_max, b->m_max) > device_smem_optin())
    return set_error(CS_EUNSUPPORTED,
                     "nv_max = %d with m_max = %d needs %zu bytes of shared memory per CTA "
                     "(limit %zu)",
                     b->nv_max, b->m_max, cta_smem_bytes(b->nv_max, b->m_max),
                     device_smem_optin());
  return CS_OK;
}

int check_batch_shapes(const cs_batch* b, const cs_options* o) {
  if (!b || !o) return set_error(CS_EINVAL, "batch and options must not be NULL");
  if (b->n < 0) return set_error(CS_EINVAL, "n = %d < 0", b->n);
  if (b->n == 0) return CS_OK;
  if (b->nv_max < 1 || b->nv_max > 128)
    return set_error(CS_EUNSUPPORTED, "nv_max = %d outside 1..128", b->nv_max);
  if (b->m_max < 0 || b->m_max > 1024)
    return set_error(CS_EUNSUPPORTED, "m_max = %d outside 0..1024", b->m_max);
  if (!b->inst || !b->M || !b->qfrc)
    return set_error(CS_EINVAL, "inst, M and qfrc must not be NULL");
  if (b->m_max > 0 && (!b->J || !b->aref || !b->D))
    return set_error(CS_EINVAL, "J, aref and D must not be NULL when m_max > 0");
  if (b->total_M < 0 || b->total_J < 0 || b->total_v < 0 || b->total_r < 0)
    return set_error(CS_EINVAL, "negative array totals");
  if (!(o->tol >= 0.f)) return set_error(CS_EINVAL, "tol must be >= 0");
  if (o->max_iter < 0 || o->max_iter > 100000)
    return set_error(CS_EINVAL, "max_iter = %d outside 0..100000", o->max_iter);
  if (o->warps_per_block < 0 || o->warps_per_block > 8)
    return set_error(CS_EINVAL, "warps_per_block = %d outside 0..8", o->warps_per_block);
  return CS_OK;
}

csk::Params make_params(const cs_batch* b, const cs_options* o) {
  csk::Params P;
  memset(&P, 0, sizeof(P));
  P.n = b->n;
  P.n_work = b->n;
  P.inst = b->inst;
  P.M = b->M;
  P.J = b->J;
  P.qfrc = b->qfrc;
  P.aref = b->aref;
  P.D = b->D;
  P.total_M = b->total_M;
  P.total_J = b->total_J;
  P.total_v = b->total_v;
  P.total_r = b->total_r;
  P.tol = o->tol;
  P.max_iter = o->max_iter;
  P.keep_factor = o->keep_factor;
  return P;
}

}  // namespace cs

using namespace cs;

extern "C" {

int cs_version(void) { return 100; }

const char* cs_strerror(int code) {
  switch (code) {
    case CS_OK: return "ok";
    case CS_EINVAL: return "invalid argument";
    case CS_ECUDA: return "CUDA error";
    case CS_ENOMEM: return "out of memory";
    case CS_EBUSY: return "busy: no free slot or arena space";
    case CS_ENOTFOUND: return "unknown ticket";
    case CS_EUNSUPPORTED: return "unsupported size";
    case CS_PENDING: return "pending";
    default: return "unknown error code";
  }
}

const char* cs_last_error(void) { return g_last_error; }

int cs_solve_fwd(const cs_batch* batch, const cs_options* opt, float* a, const cs_state* st,
                 void* stream) {
  int rc = check_batch(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (!a || !st || !st->a_lo || !st->status || !st->iters || (batch->m_max > 0 && !st->act))
    return set_error(CS_EINVAL, "a and the state arrays must not be NULL");
  csk::Params P = make_params(batch, opt);
  P.a = a;
  P.a_lo = st->a_lo;
  P.act = st->act;
  P.Lst = opt->keep_factor ? st->L : nullptr;
  P.status = st->status;
  P.iters = st->iters;
  LaunchCfg cfg;
  cfg.warps_per_block = opt->warps_per_block;
  cudaError_t e = launch_dispatch(csk::MODE_FWD, batch->nv_max, batch->m_max, P, cfg,
                                  (cudaStream_t)stream, nullptr);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_fwd launch");
}

int cs_solve_adjoint(const cs_batch* batch, const cs_options* opt, const float* a,
                     const cs_state* st, const float* g, float* dqfrc, float* daref, float* dJ,
                     void* stream) {
  return cs_solve_adjoint_theta(batch, opt, a, st, g, dqfrc, daref, dJ, nullptr, nullptr,
                                stream);
}

int cs_solve_adjoint_theta(const cs_batch* batch, const cs_options* opt, const float* a,
                           const cs_state* st, const float* g, float* dqfrc, float* daref,
                           float* dJ, float* dM, float* dD, void* stream) {
  int rc = check_batch(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (!a || !st || !st->a_lo || !st->status || !st->iters || !g || !dqfrc ||
      (batch->m_max > 0 && (!st->act || !daref || !dJ)))
    return set_error(CS_EINVAL, "a, g, the outputs and the state arrays must not be NULL");
  csk::Params P = make_params(batch, opt);
  P.a = const_cast<float*>(a);
  P.g = g;
  P.a_lo = st->a_lo;
  P.act = st->act;
  P.Lst = opt->keep_factor ? st->L : nullptr;
  P.status = st->status;
  P.iters = st->iters;
  P.dqfrc = dqfrc;
  P.daref = daref;
  P.dJ = dJ;
  P.dM = dM;
  P.dD = batch->m_max > 0 ? dD : nullptr;
  LaunchCfg cfg;
  cfg.warps_per_block = opt->warps_per_block;
  cudaError_t e = launch_dispatch(csk::MODE_ADJ, batch->nv_max, batch->m_max, P, cfg,
                                  (cudaStream_t)stream, nullptr);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_adjoint launch");
}

// ---- library-owned states ------------------------------------------------

}  // extern "C"

namespace {

// A state the library allocated: the public struct first (its address is the
// handle the caller holds), then what the library needs to check and free it.
struct OwnedState {
  cs_state pub;
  int32_t n;
  int64_t total_M, total_v, total_r;
  int32_t keep_factor;
  void* mem;
};

std::mutex g_owned_mu;
std::set<const cs_state*> g_owned;

OwnedState* owned(const cs_state* st) {
  std::lock_guard<std::mutex> lk(g_owned_mu);
  if (!st || !g_owned.count(st)) return nullptr;
  return reinterpret_cast<OwnedState*>(const_cast<cs_state*>(st));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int cs_state_create(const cs_batch* batch, int32_t keep_factor, cs_state** out) {
  if (!out) return set_error(CS_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (!batch) return set_error(CS_EINVAL, "batch must not be NULL");
  if (batch->n < 0 || batch->total_M < 0 || batch->total_v < 0 || batch->total_r < 0)
    return set_error(CS_EINVAL, "negative batch size or totals");
  if (keep_factor != 0 && keep_factor != 1)
    return set_error(CS_EINVAL, "keep_factor must be 0 or 1");
  const size_t n = (size_t)batch->n;
  const size_t b_alo = align256(4 * (size_t)batch->total_v);
  const size_t b_act = align256((size_t)batch->total_r);
  const size_t b_L = keep_factor ? align256(4 * (size_t)batch->total_M) : 0;
  const size_t b_st = align256(4 * n);
  const size_t total = b_alo + b_act + b_L + 2 * b_st;
  OwnedState* o = new (std::nothrow) OwnedState();
  if (!o) return set_error(CS_ENOMEM, "state: host allocation failed");
  o->n = batch->n;
  o->total_M = batch->total_M;
  o->total_v = batch->total_v;
  o->total_r = batch->total_r;
  o->keep_factor = keep_factor;
  o->mem = nullptr;
  if (total > 0) {
    cudaError_t e = cudaMalloc(&o->mem, total);
    if (e != cudaSuccess) {
      delete o;
      return set_error(CS_ENOMEM, "state: %s", cudaGetErrorString(e));
    }
  }
  char* cur = (char*)o->mem;
  o->pub.a_lo = (float*)cur;
  cur += b_alo;
  o->pub.act = (uint8_t*)cur;
  cur += b_act;
  o->pub.L = keep_factor ? (float*)cur : nullptr;
  cur += b_L;
  o->pub.status = (int32_t*)cur;
  cur += b_st;
  o->pub.iters = (int32_t*)cur;
  {
    std::lock_guard<std::mutex> lk(g_owned_mu);
    g_owned.insert(&o->pub);
  }
  *out = &o->pub;
  return CS_OK;
}

void cs_state_free(cs_state* st) {
  OwnedState* o = owned(st);
  if (!o) return;
  {
    std::lock_guard<std::mutex> lk(g_owned_mu);
    g_owned.erase(st);
  }
  if (o->mem) cudaFree(o->mem);
  delete o;
}

int cs_solve_fwd_alloc(const cs_batch* batch, const cs_options* opt, float* a, cs_state** st,
                       void* stream) {
  if (!st) return set_error(CS_EINVAL, "st must not be NULL");
  int rc = check_batch(batch, opt);
  if (rc != CS_OK) return rc;
  bool created = false;
  if (!*st) {
    rc = cs_state_create(batch, opt->keep_factor ? 1 : 0, st);
    if (rc != CS_OK) return rc;
    created = true;
  } else {
    const OwnedState* o = owned(*st);
    if (!o) return set_error(CS_EINVAL, "*st is not a state made by cs_state_create");
    if (o->n != batch->n || o->total_M != batch->total_M || o->total_v != batch->total_v ||
        o->total_r != batch->total_r)
      return set_error(CS_EINVAL, "the state was made for a batch of other sizes");
    if (opt->keep_factor && !o->keep_factor)
      return set_error(CS_EINVAL, "keep_factor is 1 but the state has no factor array");
  }
  rc = cs_solve_fwd(batch, opt, a, *st, stream);
  if (rc != CS_OK && created) {
    cs_state_free(*st);
    *st = nullptr;
  }
  return rc;
}

int cs_state_status(const cs_state* st, int32_t* status, int32_t* iters, void* stream) {
  const OwnedState* o = owned(st);
  if (!o) return set_error(CS_EINVAL, "not a state made by cs_state_create");
  if (o->n == 0) return CS_OK;
  const size_t bytes = 4 * (size_t)o->n;
  cudaStream_t s = (cudaStream_t)stream;
  if (status) {
    cudaError_t e = cudaMemcpyAsync(status, o->pub.status, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "cs_state_status");
  }
  if (iters) {
    cudaError_t e = cudaMemcpyAsync(iters, o->pub.iters, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "cs_state_status");
  }
  return CS_OK;
}

size_t cs_fused_workspace_bytes(int32_t n) {
  (void)n;
  return 256;
}

int cs_solve_fused(const cs_batch* batch, const cs_options* opt, const float* g,
                   const int32_t* order, float* a, float* dqfrc, float* daref, float* dJ,
                   int32_t* status, int32_t* iters, void* workspace, size_t workspace_bytes,
                   void* stream) {
  return cs_solve_fused_theta(batch, opt, g, order, a, dqfrc, daref, dJ, nullptr, nullptr,
                              status, iters, workspace, workspace_bytes, stream);
}

int cs_solve_fused_ncg(const cs_batch* batch, const cs_options* opt, const float* g,
                       const int32_t* order, float* a, float* dqfrc, float* daref, float* dJ,
                       int32_t* status, int32_t* iters, void* workspace, size_t workspace_bytes,
                       void* stream) {
  int rc = check_batch_shapes(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (!uses_warp_kernel(batch->nv_max, batch->m_max))
    return set_error(CS_EUNSUPPORTED,
                     "the conjugate-gradient solve runs one warp per instance: nv_max <= 32 "
                     "and m_max <= 256 (got %d, %d)",
                     batch->nv_max, batch->m_max);
  if (!g || !a || !dqfrc || !status || !iters || (batch->m_max > 0 && (!daref || !dJ)))
    return set_error(CS_EINVAL, "g and the output arrays must not be NULL");
  if (!workspace || workspace_bytes < cs_fused_workspace_bytes(batch->n) ||
      (reinterpret_cast<uintptr_t>(workspace) & 15))
    return set_error(CS_EINVAL, "workspace must be >= %zu bytes and 16-byte aligned",
                     cs_fused_workspace_bytes(batch->n));
  csk::Params P = make_params(batch, opt);
  P.g = g;
  P.a = a;
  P.dqfrc = dqfrc;
  P.daref = daref;
  P.dJ = dJ;
  P.status = status;
  P.iters = iters;
  P.counter = reinterpret_cast<int32_t*>(workspace);
  P.order = order;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused_ncg counter reset");
  LaunchCfg cfg;
  cfg.warps_per_block = opt->warps_per_block;
  e = launch_warp(csk::MODE_FUSED_NCG, batch->nv_max, batch->m_max, P, cfg, s, nullptr);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_fused_ncg launch");
}

int cs_solve_fused_theta(const cs_batch* batch, const cs_options* opt, const float* g,
                         const int32_t* order, float* a, float* dqfrc, float* daref, float* dJ,
                         float* dM, float* dD, int32_t* status, int32_t* iters,
                         void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_batch(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (!g || !a || !dqfrc || !status || !iters || (batch->m_max > 0 && (!daref || !dJ)))
    return set_error(CS_EINVAL, "g and the output arrays must not be NULL");
  if (!workspace || workspace_bytes < cs_fused_workspace_bytes(batch->n) ||
      (reinterpret_cast<uintptr_t>(workspace) & 15))
    return set_error(CS_EINVAL, "workspace must be >= %zu bytes and 16-byte aligned",
                     cs_fused_workspace_bytes(batch->n));
  csk::Params P = make_params(batch, opt);
  P.g = g;
  P.a = a;
  P.dqfrc = dqfrc;
  P.daref = daref;
  P.dJ = dJ;
  P.dM = dM;
  P.dD = batch->m_max > 0 ? dD : nullptr;
  P.status = status;
  P.iters = iters;
  P.counter = reinterpret_cast<int32_t*>(workspace);
  P.order = order;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused counter reset");
  LaunchCfg cfg;
  cfg.warps_per_block = opt->warps_per_block;
  e = launch_dispatch(csk::MODE_FUSED, batch->nv_max, batch->m_max, P, cfg, s, nullptr);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_fused launch");
}

}  // extern "C"
