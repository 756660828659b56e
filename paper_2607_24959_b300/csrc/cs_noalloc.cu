// cs_noalloc.cu -- the fused solve for callers that cannot allocate device
// memory (no cudaMalloc in their process, a pre-sized memory pool owned by a
// host framework, or a context in which allocation is forbidden).
//
// cs_solve_fused needs a small scratch workspace (the claim counter, and the
// claim order a plan uploads).  This variant keeps that scratch in a
// file-scope device array instead, so the call itself allocates nothing: the
// array is part of the library image and every GPU that loads the library
// holds it until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "contact_solve.h"
#include "cs_host.h"
#include "cs_warp.cuh"

namespace cs {
namespace {

// Scratch: 64 words of claim counter (a 256-byte line of its own), then the
// claim order, one int32 per instance.
constexpr int32_t kCounterWords = 64;
static __device__ __align__(256) int32_t g_static_scratch[kCounterWords + CS_STATIC_MAX_INSTANCES];

// Device address of g_static_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and passed to the kernel.
std::mutex g_addr_mu;
int32_t* g_addr[64] = {};

int scratch_address(int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused_static: cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(CS_EUNSUPPORTED, "device ordinal %d >= 64", dev);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused_static: cudaGetSymbolAddress");
    g_addr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_addr[dev];
  return CS_OK;
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" int cs_solve_fused_static(const cs_batch* batch, const cs_options* opt,
                                     const float* g, const cs_inst* inst_host, float* a,
                                     float* dqfrc, float* daref, float* dJ, int32_t* status,
                                     int32_t* iters, void* stream) {
  int rc = check_batch(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (batch->n > CS_STATIC_MAX_INSTANCES)
    return set_error(CS_EUNSUPPORTED,
                     "cs_solve_fused_static: n = %d exceeds the static scratch capacity of %d "
                     "instances; use cs_solve_fused with a workspace",
                     batch->n, (int)CS_STATIC_MAX_INSTANCES);
  if (!g || !a || !dqfrc || !status || !iters || (batch->m_max > 0 && (!daref || !dJ)))
    return set_error(CS_EINVAL, "g and the output arrays must not be NULL");
  int32_t* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != CS_OK) return rc;
  int32_t* counter = scratch;
  int32_t* order = scratch + kCounterWords;
  cudaStream_t s = (cudaStream_t)stream;
  if (inst_host) {
    // the claim order is uploaded from a host vector that lives only for the
    // call: a stream being captured would record a copy from freed memory
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return cuda_error(ce, "cs_solve_fused_static: cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
      return set_error(CS_EUNSUPPORTED,
                       "cs_solve_fused_static: cost-ordered claims (inst_host != NULL) upload "
                       "a host array and cannot be captured; pass inst_host = NULL");
    // most expensive instances are claimed first (m nv^2 + nv^3)
    std::vector<std::pair<double, int32_t>> cost(batch->n);
    for (int32_t i = 0; i < batch->n; ++i) {
      const double nv = inst_host[i].nv > 0 ? inst_host[i].nv : 1;
      const double m = inst_host[i].m > 0 ? inst_host[i].m : 0;
      cost[i] = {m * nv * nv + nv * nv * nv, i};
    }
    std::stable_sort(cost.begin(), cost.end(),
                     [](const std::pair<double, int32_t>& x, const std::pair<double, int32_t>& y) {
                       return x.first > y.first;
                     });
    std::vector<int32_t> h(batch->n);
    for (int32_t i = 0; i < batch->n; ++i) h[i] = cost[i].second;
    // from pageable memory: returns once the data are staged, so h may go
    cudaError_t e = cudaMemcpyAsync(order, h.data(), h.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused_static: order upload");
  }
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused_static: counter reset");
  csk::Params P = make_params(batch, opt);
  P.g = g;
  P.a = a;
  P.dqfrc = dqfrc;
  P.daref = daref;
  P.dJ = dJ;
  P.status = status;
  P.iters = iters;
  P.counter = counter;
  P.order = inst_host ? order : nullptr;
  LaunchCfg cfg;
  cfg.warps_per_block = opt->warps_per_block;
  e = launch_dispatch(csk::MODE_FUSED, batch->nv_max, batch->m_max, P, cfg, s, nullptr);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_fused_static launch");
}
