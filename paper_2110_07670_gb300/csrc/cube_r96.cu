// cube_r96.cu -- the pair passes' compile-time kernels on the 96^3 box for the
// alternative radix plans the autotuner times (8 x 12, 16 x 6).
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"

namespace ace {

template cudaError_t pass_detail::dispatch_cube<96, 8>(const PassArgs&, const PassShape&, int, int, int, int,
                                                    int, cudaStream_t);
template cudaError_t zline_launch<96, 8>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<96, 8>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pipeline_launch<96, 8>(const PassArgs&, const PipeArgs&, cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<96, 16>(const PassArgs&, const PassShape&, int, int, int, int,
                                                    int, cudaStream_t);
template cudaError_t zline_launch<96, 16>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<96, 16>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pipeline_launch<96, 16>(const PassArgs&, const PipeArgs&, cudaStream_t);

}  // namespace ace
