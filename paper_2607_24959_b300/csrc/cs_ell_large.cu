// cs_ell_large.cu -- round-cone kernels for nv <= 18 and <= 32.
#include "cs_ell_launch.cuh"

namespace cs {
template cudaError_t launch_ell_nv<18>(int, const csk::EParams&, const LaunchCfg&, cudaStream_t);
template cudaError_t launch_ell_nv<32>(int, const csk::EParams&, const LaunchCfg&, cudaStream_t);
}  // namespace cs
