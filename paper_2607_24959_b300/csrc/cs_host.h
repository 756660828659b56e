// cs_host.h -- internal host-side declarations shared by the library's .cu
// files (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

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
