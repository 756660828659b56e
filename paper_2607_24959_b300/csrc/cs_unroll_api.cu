// cs_unroll_api.cu -- C entry points of the unrolled-differentiation
// comparison path (forward with trace, reverse sweep): one warp per instance
// for nv <= 32 and m <= 256, one CTA per instance beyond.
#include <cuda_runtime.h>

#include "contact_solve.h"
#include "cs_host.h"
#include "cs_unrolled.cuh"

namespace cs {

template <int NV>
cudaError_t launch_unrolled_nv(int dir, int mt, const csk::UParams& U, cudaStream_t s);
extern template cudaError_t launch_unrolled_nv<3>(int, int, const csk::UParams&, cudaStream_t);
extern template cudaError_t launch_unrolled_nv<9>(int, int, const csk::UParams&, cudaStream_t);
extern template cudaError_t launch_unrolled_nv<18>(int, int, const csk::UParams&, cudaStream_t);
extern template cudaError_t launch_unrolled_nv<32>(int, int, const csk::UParams&, cudaStream_t);
cudaError_t launch_unrolled_cta(int dir, int nv_max, int m_max, const csk::UParams& U,
                                cudaStream_t s);
size_t cta_unrolled_smem_bytes(int nv_max, int m_max);

namespace {

int64_t slot_floats(const cs_batch* b) {
  return b->total_M + 4 * b->total_v + 2 * (int64_t)b->n;
}

int check_unrolled(const cs_batch* b, const cs_options* o) {
  int rc = check_batch_shapes(b, o);
  if (rc != CS_OK || b->n == 0) return rc;
  if (!uses_warp_kernel(b->nv_max, b->m_max) &&
      cta_unrolled_smem_bytes(b->nv_max, b->m_max) > device_smem_optin())
    return set_error(CS_EUNSUPPORTED,
                     "unrolled differentiation: nv_max = %d with m_max = %d needs %zu bytes of "
                     "shared memory per CTA (limit %zu)",
                     b->nv_max, b->m_max, cta_unrolled_smem_bytes(b->nv_max, b->m_max),
                     device_smem_optin());
  return CS_OK;
}

cudaError_t launch_unrolled(int dir, const cs_batch* b, const csk::UParams& U, cudaStream_t s) {
  if (!uses_warp_kernel(b->nv_max, b->m_max))
    return launch_unrolled_cta(dir, b->nv_max, b->m_max, U, s);
  const int nvb = nv_bucket(b->nv_max), mt = mt_bucket(b->m_max);
  switch (nvb) {
    case 3: return launch_unrolled_nv<3>(dir, mt, U, s);
    case 9: return launch_unrolled_nv<9>(dir, mt, U, s);
    case 18: return launch_unrolled_nv<18>(dir, mt, U, s);
    default: return launch_unrolled_nv<32>(dir, mt, U, s);
  }
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" {

size_t cs_unrolled_trace_floats(const cs_batch* batch, int32_t K) {
  if (!batch || K < 0 || batch->n < 0) return 0;
  return (size_t)K * (size_t)slot_floats(batch);
}

size_t cs_unrolled_mask_bytes(const cs_batch* batch, int32_t K) {
  if (!batch || K < 0 || batch->total_r < 0) return 0;
  return (size_t)K * (size_t)batch->total_r;
}

int cs_unrolled_fwd(const cs_batch* batch, const cs_options* opt, float* a, float* trace,
                    uint8_t* tmask, int32_t* status, int32_t* iters, void* stream) {
  int rc = check_unrolled(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (!a || !status || !iters || (opt->max_iter > 0 && (!trace || !tmask)))
    return set_error(CS_EINVAL, "a, status, iters and (for K > 0) the trace must not be NULL");
  csk::UParams U;
  U.P = make_params(batch, opt);
  U.P.a = a;
  U.P.status = status;
  U.P.iters = iters;
  U.trace = trace;
  U.tmask = tmask;
  U.slot = slot_floats(batch);
  cudaError_t e = launch_unrolled(0, batch, U, (cudaStream_t)stream);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_unrolled_fwd launch");
}

int cs_unrolled_bwd(const cs_batch* batch, const cs_options* opt, const float* a,
                    const float* trace, const uint8_t* tmask, int32_t* status,
                    const int32_t* iters, const float* g, float* dqfrc, float* daref, float* dJ,
                    float* dM, float* dD, void* stream) {
  int rc = check_unrolled(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  if (!a || !status || !iters || !g || !dqfrc || !dM ||
      (batch->m_max > 0 && (!daref || !dJ || !dD)) ||
      (opt->max_iter > 0 && (!trace || !tmask)))
    return set_error(CS_EINVAL, "a, the trace, status, iters, g and the outputs must not be NULL");
  csk::UParams U;
  U.P = make_params(batch, opt);
  U.P.a = const_cast<float*>(a);
  U.P.status = status;
  U.P.iters = const_cast<int32_t*>(iters);
  U.P.g = g;
  U.P.dqfrc = dqfrc;
  U.P.daref = daref;
  U.P.dJ = dJ;
  U.P.dM = dM;
  U.P.dD = dD;
  U.trace = const_cast<float*>(trace);
  U.tmask = const_cast<uint8_t*>(tmask);
  U.slot = slot_floats(batch);
  cudaError_t e = launch_unrolled(1, batch, U, (cudaStream_t)stream);
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_unrolled_bwd launch");
}

}  // extern "C"
