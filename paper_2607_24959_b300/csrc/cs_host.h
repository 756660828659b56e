// cs_host.h -- internal host-side declarations shared by the library's .cu
// files (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "contact_solve.h"

namespace csk {
struct Params;
}

namespace cs {

// Launch geometry of the warp-per-instance kernels.
struct LaunchCfg {
  int warps_per_block = 0;  // 0: default (4)
  int blocks_per_sm = 0;    // 0: as many as fit
};

// What a launch used (for the autotuner and reports).
struct KernelInfo {
  int nv_bucket = 0, mt = 0, warps_per_block = 0, grid = 0, smem_bytes = 0,
      blocks_per_sm = 0;
};

int set_error(int code, const char* fmt, ...);

// Launch set-up of one kernel, done once per device and shape: the dynamic
// shared-memory attribute (raised when a larger size is asked for) and the
// resident blocks per SM of each (block size, shared memory).  A launch
// pays for these runtime queries only the first time (they cost tens of
// microseconds, which a serving batch of small instances would pay per
// bucket launch).
struct KernelSetup {
  std::mutex mu;
  size_t smem_set[16] = {};
  std::map<std::tuple<int, int, size_t>, int> per_sm;
};

template <class Kernel>
cudaError_t kernel_setup(KernelSetup& ks, Kernel kern, int threads, size_t smem, int* per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(ks.mu);
  const bool cached = dev >= 0 && dev < 16;
  if (!cached || ks.smem_set[dev] < smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // all of the unified L1/shared array as shared memory: the warps' (or
    // CTAs') slices are the working set, and occupancy hides the latency
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (cached) ks.smem_set[dev] = smem;
  }
  const auto key = std::make_tuple(dev, threads, smem);
  auto it = ks.per_sm.find(key);
  if (it != ks.per_sm.end()) {
    *per_sm = it->second;
    return cudaSuccess;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem);
  if (e == cudaSuccess) ks.per_sm[key] = *per_sm;
  return e;
}
int cuda_error(cudaError_t e, const char* where);
int nv_bucket(int nv);
int mt_bucket(int m);
int device_sm_count();
size_t device_smem_optin();

// Per-nv-bucket launchers (one translation unit each, compiled in parallel).
template <int NV>
cudaError_t launch_nv(int mode, int mt, const csk::Params& P, const LaunchCfg& cfg,
                      cudaStream_t s, KernelInfo* info);
extern template cudaError_t launch_nv<3>(int, int, const csk::Params&, const LaunchCfg&,
                                         cudaStream_t, KernelInfo*);
extern template cudaError_t launch_nv<9>(int, int, const csk::Params&, const LaunchCfg&,
                                         cudaStream_t, KernelInfo*);
extern template cudaError_t launch_nv<18>(int, int, const csk::Params&, const LaunchCfg&,
                                          cudaStream_t, KernelInfo*);
extern template cudaError_t launch_nv<32>(int, int, const csk::Params&, const LaunchCfg&,
                                          cudaStream_t, KernelInfo*);
// One CTA per instance (nv > 32 or m > 256; nv <= 128, m <= 1024).
int cta_rows_per_thread(int m_max);
size_t cta_smem_bytes(int nv_max, int m_max);
cudaError_t launch_cta(int mode, int nv_max, int m_max, const csk::Params& P, cudaStream_t s,
                       KernelInfo* info);
// Warp kernels when nv_max <= 32 and m_max <= 256, else the CTA kernels.
bool uses_warp_kernel(int nv_max, int m_max);
cudaError_t launch_dispatch(int mode, int nv_max, int m_max, const csk::Params& P,
                            const LaunchCfg& cfg, cudaStream_t s, KernelInfo* info);
int launch_error(cudaError_t e, const char* where);
// Argument, shape and option checks; check_batch also checks that a batch
// solved by one CTA kernel fits its shared memory (plans check per bucket).
int check_batch(const cs_batch* b, const cs_options* o);
int check_batch_shapes(const cs_batch* b, const cs_options* o);
csk::Params make_params(const cs_batch* b, const cs_options* o);
cudaError_t launch_warp(int mode, int nv_max, int m_max, const csk::Params& P,
                        const LaunchCfg& cfg, cudaStream_t s, KernelInfo* info);

}  // namespace cs
