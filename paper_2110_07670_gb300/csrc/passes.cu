// passes.cu -- generic (runtime-geometry) pass kernels and the dispatch that
// prefers the compile-time cube kernels when the box is one of their sizes.
#include "pass_kernel.cuh"

namespace ace {

template <typename R>
cudaError_t launch_pass(const PassArgs& a0, const PassShape& s, int pro, int epi, int mid, int sgn, int batch,
                        cudaStream_t st) {
    PassArgs a = a0;
    a.tz = s.tz;
    a.ty = s.ty;
    a.tx = s.tx;
    a.axes = s.axes;
    a.bulk = s.bulk;
    a.vec = s.vec;
    if (batch <= 0) return cudaSuccess;
    // runtime-geometry kernels are bounded at 512 threads, compile-time cubes at their own count
    if (s.threads > (s.cube ? 1024 : 512) || (s.threads & 31)) return cudaErrorInvalidConfiguration;
    if (s.cube) {
        if (sizeof(R) != 4 || a.n0 != a.n1 || a.n1 != a.n2) return cudaErrorInvalidValue;
        return cube_pass_launch(a.n0, a, s, pro, epi, mid, sgn, batch, st);
    }
    return pass_detail::dispatch<pass_detail::DynShape, R>(a, s, pro, epi, mid, sgn, batch, st);
}

template cudaError_t launch_pass<float>(const PassArgs&, const PassShape&, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_pass<double>(const PassArgs&, const PassShape&, int, int, int, int, int, cudaStream_t);

}  // namespace ace
