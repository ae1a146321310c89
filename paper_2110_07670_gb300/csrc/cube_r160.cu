// cube_r160.cu -- the pair passes' compile-time kernels on the 160^3 box for the
// alternative radix plans the autotuner times (10 x 16).
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"

namespace ace {

template cudaError_t pass_detail::dispatch_cube<160, 10>(const PassArgs&, const PassShape&, int, int, int, int,
                                                    int, cudaStream_t);
template cudaError_t zline_launch<160, 10>(const PassArgs&, int, cudaStream_t);
template cudaError_t tplane_launch<160, 10>(int, const PassArgs&, int, cudaStream_t);
template cudaError_t pipeline_launch<160, 10>(const PassArgs&, const PipeArgs&, cudaStream_t);

}  // namespace ace
