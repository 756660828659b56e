// cs_ell_cta.cu -- instantiates and launches the one-CTA-per-instance
// round-cone kernels (instances with nv > 32 or m > 256).
#include "cs_cta_elliptic.cuh"
#include "cs_host.h"

namespace cs {

size_t cta_elliptic_smem_bytes(int nv_max, int m_max) {
  return csk::CtaEllGeo::make(nv_max, m_max).bytes();
}

template <int MTC>
static cudaError_t launch_ell_cta_t(int nv_max, int m_max, const csk::EParams& EP,
                                    cudaStream_t s) {
  auto kern = csk::cta_elliptic_kernel<MTC>;
  const csk::CtaEllGeo eg = csk::CtaEllGeo::make(nv_max, m_max);
  const size_t smem = eg.bytes();
  if (smem > device_smem_optin()) return cudaErrorInvalidConfiguration;
  static KernelSetup setup;
  int per_sm = 0;
  cudaError_t e = kernel_setup(setup, kern, csk::kCtaThreads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * device_sm_count();
  if (grid > EP.P.n_work) grid = EP.P.n_work;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, csk::kCtaThreads, smem, s>>>(EP, eg);
  return cudaGetLastError();
}

cudaError_t launch_ell_cta(int nv_max, int m_max, const csk::EParams& EP, cudaStream_t s) {
  if (nv_max < 1 || nv_max > csk::kCtaNvMax) return cudaErrorInvalidValue;
  switch (cta_rows_per_thread(m_max)) {
    case 1: return launch_ell_cta_t<1>(nv_max, m_max, EP, s);
    case 2: return launch_ell_cta_t<2>(nv_max, m_max, EP, s);
    case 4: return launch_ell_cta_t<4>(nv_max, m_max, EP, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
