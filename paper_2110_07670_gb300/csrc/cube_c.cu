// cube_c.cu -- compile-time pass kernels for the N^3 boxes N = 108, 120, 160.
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"
#include "halfplane.cuh"

namespace ace {

template cudaError_t pass_detail::dispatch_cube<108>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<120>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);
template cudaError_t pass_detail::dispatch_cube<160>(const PassArgs&, const PassShape&, int, int, int, int, int,
                                                  cudaStream_t);

template cudaError_t zline_launch<108>(const PassArgs&, int, cudaStream_t);
template cudaError_t zline_launch<120>(const PassArgs&, int, cudaStream_t);
template cudaError_t zline_launch<160>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<160>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pipeline_launch<160>(const PassArgs&, const PipeArgs&, cudaStream_t);
template cudaError_t tplane_launch<108>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<120>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t halfplane_launch<120>(int, const PassArgs&, int, cudaStream_t);

}  // namespace ace
