// cs_kern_nv18.cu -- instantiates the warp-per-instance kernels for nv <= 18.
#include "cs_launch.cuh"

namespace cs {
template cudaError_t launch_nv<18>(int, int, const csk::Params&, const LaunchCfg&,
                                    cudaStream_t, KernelInfo*);
}  // namespace cs
