// cs_unroll_large.cu -- unrolled-differentiation kernels for nv <= 18 and <= 32.
#include "cs_unroll_launch.cuh"

namespace cs {
template cudaError_t launch_unrolled_nv<18>(int, int, const csk::UParams&, cudaStream_t);
template cudaError_t launch_unrolled_nv<32>(int, int, const csk::UParams&, cudaStream_t);
}  // namespace cs
