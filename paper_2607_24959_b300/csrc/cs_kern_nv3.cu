// cs_kern_nv3.cu -- instantiates the warp-per-instance kernels for nv <= 3.
#include "cs_launch.cuh"

namespace cs {
template cudaError_t launch_nv<3>(int, int, const csk::Params&, const LaunchCfg&,
                                    cudaStream_t, KernelInfo*);
}  // namespace cs
