// cs_ell_launch.cuh -- launch geometry of the round-cone kernels (one warp
// per instance).  Included by cs_ell_*.cu only.
#pragma once

#include "cs_elliptic.cuh"
#include "cs_host.h"

namespace cs {

template <int NV, int MT>
static cudaError_t launch_ell_t(const csk::EParams& EP, const LaunchCfg& cfg, cudaStream_t s) {
  using E = csk::EGeo<NV, MT>;
  auto kern = csk::warp_elliptic_kernel<NV, MT>;
  int wpb = cfg.warps_per_block > 0 ? cfg.warps_per_block : 4;
  if (wpb > 8) wpb = 8;
  const size_t optin = device_smem_optin();
  while (wpb > 1 && (size_t)wpb * E::kBytes > optin) --wpb;
  const size_t smem = (size_t)wpb * E::kBytes;
  static KernelSetup setup;
  int per_sm = 0;
  cudaError_t e = kernel_setup(setup, kern, wpb * 32, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)per_sm * device_sm_count();
  const long long need = ((long long)EP.P.n_work + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, wpb * 32, smem, s>>>(EP);
  return cudaGetLastError();
}

template <int NV>
cudaError_t launch_ell_nv(int mt, const csk::EParams& EP, const LaunchCfg& cfg, cudaStream_t s) {
  switch (mt) {
    case 1: return launch_ell_t<NV, 1>(EP, cfg, s);
    case 2: return launch_ell_t<NV, 2>(EP, cfg, s);
    case 3: return launch_ell_t<NV, 3>(EP, cfg, s);
    case 4: return launch_ell_t<NV, 4>(EP, cfg, s);
    case 6: return launch_ell_t<NV, 6>(EP, cfg, s);
    case 8: return launch_ell_t<NV, 8>(EP, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cs
