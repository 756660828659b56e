// cs_unroll_small.cu -- unrolled-differentiation kernels for nv <= 3 and <= 9.
#include "cs_unroll_launch.cuh"

namespace cs {
template cudaError_t launch_unrolled_nv<3>(int, int, const csk::UParams&, cudaStream_t);
template cudaError_t launch_unrolled_nv<9>(int, int, const csk::UParams&, cudaStream_t);
}  // namespace cs
