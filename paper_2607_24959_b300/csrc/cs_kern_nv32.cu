// cs_kern_nv32.cu -- instantiates the warp-per-instance kernels for nv <= 32.
#include "cs_launch.cuh"

namespace cs {
template cudaError_t launch_nv<32>(int, int, const csk::Params&, const LaunchCfg&,
                                    cudaStream_t, KernelInfo*);
}  // namespace cs
