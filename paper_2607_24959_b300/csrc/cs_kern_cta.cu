// cs_kern_cta.cu -- instantiates and launches the one-CTA-per-instance
// kernels (instances with nv > 32 or m > 256).
#include "cs_cta.cuh"
#include "cs_host.h"

namespace cs {

int cta_rows_per_thread(int m_max) {
  if (m_max <= csk::kCtaThreads) return 1;
  if (m_max <= 2 * csk::kCtaThreads) return 2;
  if (m_max <= 4 * csk::kCtaThreads) return 4;
  return -1;
}

size_t cta_smem_bytes(int nv_max, int m_max) {
  return csk::CtaGeo::make(nv_max, m_max).bytes();
}

template <int MTC, int MODE>
static cudaError_t launch_cta_t(int nv_max, int m_max, const csk::Params& P, cudaStream_t s,
                                KernelInfo* info) {
  auto kern = csk::cta_solve_kernel<MTC, MODE>;
  const csk::CtaGeo geo = csk::CtaGeo::make(nv_max, m_max);
  const size_t smem = geo.bytes();
  if (smem > device_smem_optin()) return cudaErrorInvalidConfiguration;
  static KernelSetup setup;
  int per_sm = 0;
  cudaError_t e = kernel_setup(setup, kern, csk::kCtaThreads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * device_sm_count();
  if (grid > P.n_work) grid = P.n_work;
  if (grid < 1) grid = 1;
  if (info) {
    info->nv_bucket = geo.nvcap;
    info->mt = MTC;
    info->warps_per_block = csk::kCtaWarps;
    info->grid = (int)grid;
    info->smem_bytes = (int)smem;
    info->blocks_per_sm = per_sm;
  }
  kern<<<(unsigned)grid, csk::kCtaThreads, smem, s>>>(P, geo);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_cta_m(int nv_max, int m_max, const csk::Params& P, cudaStream_t s,
                                KernelInfo* info) {
  switch (cta_rows_per_thread(m_max)) {
    case 1: return launch_cta_t<1, MODE>(nv_max, m_max, P, s, info);
    case 2: return launch_cta_t<2, MODE>(nv_max, m_max, P, s, info);
    case 4: return launch_cta_t<4, MODE>(nv_max, m_max, P, s, info);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cta(int mode, int nv_max, int m_max, const csk::Params& P, cudaStream_t s,
                       KernelInfo* info) {
  if (nv_max < 1 || nv_max > csk::kCtaNvMax) return cudaErrorInvalidValue;
  switch (mode) {
    case csk::MODE_FWD: return launch_cta_m<csk::MODE_FWD>(nv_max, m_max, P, s, info);
    case csk::MODE_ADJ: return launch_cta_m<csk::MODE_ADJ>(nv_max, m_max, P, s, info);
    default: return launch_cta_m<csk::MODE_FUSED>(nv_max, m_max, P, s, info);
  }
}

}  // namespace cs
