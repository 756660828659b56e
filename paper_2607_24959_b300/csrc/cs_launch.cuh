// cs_launch.cuh -- launch geometry for the warp-per-instance kernels of one
// nv bucket.  Included by the cs_kern_nv*.cu translation units only.
#pragma once

#include "cs_host.h"
#include "cs_warp.cuh"

namespace cs {

template <int NV, int MT, int MODE>
static cudaError_t launch_t(const csk::Params& P, const LaunchCfg& cfg, cudaStream_t s,
                            KernelInfo* info) {
  using G = csk::Geo<NV, MT, true>;  // the layout warp_solve_kernel uses
  auto kern = csk::warp_solve_kernel<NV, MT, MODE>;
  int wpb = cfg.warps_per_block > 0 ? cfg.warps_per_block : 4;
  if (wpb > 8) wpb = 8;
  const size_t optin = device_smem_optin();
  while (wpb > 1 && (size_t)wpb * G::kBytes > optin) --wpb;
  const size_t smem = (size_t)wpb * G::kBytes;
  static KernelSetup setup;
  int per_sm = 0;
  cudaError_t e = kernel_setup(setup, kern, wpb * 32, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
  long long grid = (long long)per_sm * device_sm_count();
  const long long need = ((long long)P.n_work + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if (info) {
    info->nv_bucket = NV;
    info->mt = MT;
    info->warps_per_block = wpb;
    info->grid = (int)grid;
    info->smem_bytes = (int)smem;
    info->blocks_per_sm = per_sm;
  }
  kern<<<(unsigned)grid, wpb * 32, smem, s>>>(P);
  return cudaGetLastError();
}

template <int NV, int MODE>
static cudaError_t launch_mt(int mt, const csk::Params& P, const LaunchCfg& cfg,
                             cudaStream_t s, KernelInfo* info) {
  switch (mt) {
    case 1: return launch_t<NV, 1, MODE>(P, cfg, s, info);
    case 2: return launch_t<NV, 2, MODE>(P, cfg, s, info);
    case 3: return launch_t<NV, 3, MODE>(P, cfg, s, info);
    case 4: return launch_t<NV, 4, MODE>(P, cfg, s, info);
    case 6: return launch_t<NV, 6, MODE>(P, cfg, s, info);
    case 8: return launch_t<NV, 8, MODE>(P, cfg, s, info);
    default: return cudaErrorInvalidValue;
  }
}

template <int NV>
cudaError_t launch_nv(int mode, int mt, const csk::Params& P, const LaunchCfg& cfg,
                      cudaStream_t s, KernelInfo* info) {
  switch (mode) {
    case csk::MODE_FWD: return launch_mt<NV, csk::MODE_FWD>(mt, P, cfg, s, info);
    case csk::MODE_ADJ: return launch_mt<NV, csk::MODE_ADJ>(mt, P, cfg, s, info);
    case csk::MODE_FUSED_NCG: return launch_mt<NV, csk::MODE_FUSED_NCG>(mt, P, cfg, s, info);
    default: return launch_mt<NV, csk::MODE_FUSED>(mt, P, cfg, s, info);
  }
}

}  // namespace cs
