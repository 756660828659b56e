// cs_unroll_launch.cuh -- launch geometry of the unrolled-differentiation
// kernels (one warp per instance).  Included by cs_unroll_*.cu only.
#pragma once

#include "cs_host.h"
#include "cs_unrolled.cuh"

namespace cs {

template <int NV, int MT, int DIR>
static cudaError_t launch_unrolled_t(const csk::UParams& U, cudaStream_t s) {
  using G = csk::Geo<NV, MT>;
  auto kern = csk::warp_unrolled_kernel<NV, MT, DIR>;
  int wpb = 4;
  const size_t optin = device_smem_optin();
  while (wpb > 1 && (size_t)wpb * G::kBytes > optin) --wpb;
  const size_t smem = (size_t)wpb * G::kBytes;
  static KernelSetup setup;
  int per_sm = 0;
  cudaError_t e = kernel_setup(setup, kern, wpb * 32, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)per_sm * device_sm_count();
  const long long need = ((long long)U.P.n + wpb - 1) / wpb;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, wpb * 32, smem, s>>>(U);
  return cudaGetLastError();
}

template <int NV, int DIR>
static cudaError_t launch_unrolled_mt(int mt, const csk::UParams& U, cudaStream_t s) {
  switch (mt) {
    case 1: return launch_unrolled_t<NV, 1, DIR>(U, s);
    case 2: return launch_unrolled_t<NV, 2, DIR>(U, s);
    case 3: return launch_unrolled_t<NV, 3, DIR>(U, s);
    case 4: return launch_unrolled_t<NV, 4, DIR>(U, s);
    case 6: return launch_unrolled_t<NV, 6, DIR>(U, s);
    case 8: return launch_unrolled_t<NV, 8, DIR>(U, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NV>
cudaError_t launch_unrolled_nv(int dir, int mt, const csk::UParams& U, cudaStream_t s) {
  return dir == 0 ? launch_unrolled_mt<NV, 0>(mt, U, s) : launch_unrolled_mt<NV, 1>(mt, U, s);
}

}  // namespace cs
