// cs_unroll_cta.cu -- instantiates and launches the one-CTA-per-instance
// unrolled-differentiation kernels (instances with nv > 32 or m > 256).
#include "cs_cta_unrolled.cuh"
#include "cs_host.h"

namespace cs {

size_t cta_unrolled_smem_bytes(int nv_max, int m_max) {
  return csk::CtaGeo::make(nv_max, m_max, csk::CU_NVEC).bytes();
}

template <int MTC, int DIR>
static cudaError_t launch_cta_unrolled_t(int nv_max, int m_max, const csk::UParams& U,
                                         cudaStream_t s) {
  auto kern = csk::cta_unrolled_kernel<MTC, DIR>;
  const csk::CtaGeo geo = csk::CtaGeo::make(nv_max, m_max, csk::CU_NVEC);
  const size_t smem = geo.bytes();
  if (smem > device_smem_optin()) return cudaErrorInvalidConfiguration;
  static KernelSetup setup;
  int per_sm = 0;
  cudaError_t e = kernel_setup(setup, kern, csk::kCtaThreads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * device_sm_count();
  if (grid > U.P.n) grid = U.P.n;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, csk::kCtaThreads, smem, s>>>(U, geo);
  return cudaGetLastError();
}

template <int DIR>
static cudaError_t launch_cta_unrolled_m(int nv_max, int m_max, const csk::UParams& U,
                                         cudaStream_t s) {
  switch (cta_rows_per_thread(m_max)) {
    case 1: return launch_cta_unrolled_t<1, DIR>(nv_max, m_max, U, s);
    case 2: return launch_cta_unrolled_t<2, DIR>(nv_max, m_max, U, s);
    case 4: return launch_cta_unrolled_t<4, DIR>(nv_max, m_max, U, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_unrolled_cta(int dir, int nv_max, int m_max, const csk::UParams& U,
                                cudaStream_t s) {
  if (nv_max < 1 || nv_max > csk::kCtaNvMax) return cudaErrorInvalidValue;
  return dir == 0 ? launch_cta_unrolled_m<0>(nv_max, m_max, U, s)
                  : launch_cta_unrolled_m<1>(nv_max, m_max, U, s);
}

}  // namespace cs
