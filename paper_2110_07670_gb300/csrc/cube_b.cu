// cube_b.cu -- compile-time pass kernels for the N^3 boxes N = 90, 96, 100.
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"

namespace ace {

template cudaError_t pass_detail::dispatch_cube<90>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<96>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<100>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);

template cudaError_t zline_launch<90>(const PassArgs&, int, cudaStream_t);
template cudaError_t zline_launch<96>(const PassArgs&, int, cudaStream_t);
template cudaError_t zline_launch<100>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<96>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pipeline_launch<96>(const PassArgs&, const PipeArgs&, cudaStream_t);
template cudaError_t tplane_launch<90>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<100>(int, const PassArgs&, int, cudaStream_t);

}  // namespace ace
