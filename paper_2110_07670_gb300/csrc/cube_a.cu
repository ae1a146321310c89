// cube_a.cu -- compile-time pass kernels for the N^3 boxes N = 32, 60, 80.
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"

namespace ace {

template cudaError_t pass_detail::dispatch_cube<32>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<60>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<80>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);

template cudaError_t zline_launch<32>(const PassArgs&, int, cudaStream_t);
template cudaError_t zline_launch<60>(const PassArgs&, int, cudaStream_t);
template cudaError_t zline_launch<80>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<32>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<80>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pipeline_launch<32>(const PassArgs&, const PipeArgs&, cudaStream_t);
template cudaError_t pipeline_launch<80>(const PassArgs&, const PipeArgs&, cudaStream_t);
template cudaError_t tplane_launch<60>(int, const PassArgs&, int, cudaStream_t);

}  // namespace ace
