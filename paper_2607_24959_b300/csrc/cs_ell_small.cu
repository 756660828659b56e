// cs_ell_small.cu -- round-cone kernels for nv <= 3 and <= 9.
#include "cs_ell_launch.cuh"

namespace cs {
template cudaError_t launch_ell_nv<3>(int, const csk::EParams&, const LaunchCfg&, cudaStream_t);
template cudaError_t launch_ell_nv<9>(int, const csk::EParams&, const LaunchCfg&, cudaStream_t);
}  // namespace cs
