// cs_kern_nv9.cu -- instantiates the warp-per-instance kernels for nv <= 9.
#include "cs_launch.cuh"

namespace cs {
template cudaError_t launch_nv<9>(int, int, const csk::Params&, const LaunchCfg&,
                                    cudaStream_t, KernelInfo*);
}  // namespace cs
