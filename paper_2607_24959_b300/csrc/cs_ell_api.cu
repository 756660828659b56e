// cs_ell_api.cu -- C entry point of the round-cone fused solve and adjoint:
// one warp per instance for nv <= 32 and m <= 256, one CTA per instance
// beyond.
#include <cuda_runtime.h>

#include "contact_solve.h"
#include "cs_elliptic.cuh"
#include "cs_host.h"

namespace cs {

template <int NV>
cudaError_t launch_ell_nv(int mt, const csk::EParams& EP, const LaunchCfg& cfg, cudaStream_t s);
extern template cudaError_t launch_ell_nv<3>(int, const csk::EParams&, const LaunchCfg&,
                                             cudaStream_t);
extern template cudaError_t launch_ell_nv<9>(int, const csk::EParams&, const LaunchCfg&,
                                             cudaStream_t);
extern template cudaError_t launch_ell_nv<18>(int, const csk::EParams&, const LaunchCfg&,
                                              cudaStream_t);
extern template cudaError_t launch_ell_nv<32>(int, const csk::EParams&, const LaunchCfg&,
                                              cudaStream_t);
cudaError_t launch_ell_cta(int nv_max, int m_max, const csk::EParams& EP, cudaStream_t s);
size_t cta_elliptic_smem_bytes(int nv_max, int m_max);

}  // namespace cs

using namespace cs;

extern "C" int cs_solve_fused_elliptic(const cs_batch* batch, const cs_options* opt,
                                       const float* mu, const float* g, const int32_t* order,
                                       float* a, float* dqfrc, float* daref, float* dJ,
                                       float* dM, float* dD, float* dmu, int32_t* status,
                                       int32_t* iters, void* workspace,
                                       size_t workspace_bytes, void* stream) {
  int rc = check_batch_shapes(batch, opt);
  if (rc != CS_OK || batch->n == 0) return rc;
  const bool warp = uses_warp_kernel(batch->nv_max, batch->m_max);
  if (!warp && cta_elliptic_smem_bytes(batch->nv_max, batch->m_max) > device_smem_optin())
    return set_error(CS_EUNSUPPORTED,
                     "round cone: nv_max = %d with m_max = %d needs %zu bytes of shared memory "
                     "per CTA (limit %zu)",
                     batch->nv_max, batch->m_max,
                     cta_elliptic_smem_bytes(batch->nv_max, batch->m_max), device_smem_optin());
  if (!g || !a || !dqfrc || !status || !iters ||
      (batch->m_max > 0 && (!daref || !dJ || !mu)))
    return set_error(CS_EINVAL, "mu, g and the output arrays must not be NULL");
  if (!workspace || workspace_bytes < cs_fused_workspace_bytes(batch->n) ||
      (reinterpret_cast<uintptr_t>(workspace) & 15))
    return set_error(CS_EINVAL, "workspace must be >= %zu bytes and 16-byte aligned",
                     cs_fused_workspace_bytes(batch->n));
  csk::EParams EP;
  EP.P = make_params(batch, opt);
  EP.P.g = g;
  EP.P.a = a;
  EP.P.dqfrc = dqfrc;
  EP.P.daref = daref;
  EP.P.dJ = dJ;
  EP.P.dM = dM;
  EP.P.dD = batch->m_max > 0 ? dD : nullptr;
  EP.P.status = status;
  EP.P.iters = iters;
  EP.P.counter = reinterpret_cast<int32_t*>(workspace);
  EP.P.order = order;
  EP.mu = mu;
  EP.dmu = batch->m_max > 0 ? dmu : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(workspace, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_error(e, "cs_solve_fused_elliptic counter reset");
  if (!warp) {
    e = launch_ell_cta(batch->nv_max, batch->m_max, EP, s);
    return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_fused_elliptic launch");
  }
  LaunchCfg cfg;
  cfg.warps_per_block = opt->warps_per_block;
  const int mt = mt_bucket(batch->m_max);
  switch (nv_bucket(batch->nv_max)) {
    case 3: e = launch_ell_nv<3>(mt, EP, cfg, s); break;
    case 9: e = launch_ell_nv<9>(mt, EP, cfg, s); break;
    case 18: e = launch_ell_nv<18>(mt, EP, cfg, s); break;
    default: e = launch_ell_nv<32>(mt, EP, cfg, s); break;
  }
  return e == cudaSuccess ? CS_OK : launch_error(e, "cs_solve_fused_elliptic launch");
}
