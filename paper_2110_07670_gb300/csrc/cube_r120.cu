// cube_r120.cu -- the pair passes' compile-time kernels on the 120^3 box for the
// alternative radix plans the autotuner times (10 x 12, 8 x 15).
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"
#include "halfplane.cuh"

namespace ace {

template cudaError_t pass_detail::dispatch_cube<120, 10>(const PassArgs&, const PassShape&, int, int, int, int,
                                                    int, cudaStream_t);
template cudaError_t zline_launch<120, 10>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<120, 10>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t halfplane_launch<120, 10>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<120, 8>(const PassArgs&, const PassShape&, int, int, int, int,
                                                    int, cudaStream_t);
template cudaError_t zline_launch<120, 8>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<120, 8>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t halfplane_launch<120, 8>(int, const PassArgs&, int, cudaStream_t);

}  // namespace ace
