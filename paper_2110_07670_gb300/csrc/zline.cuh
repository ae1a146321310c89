// zline.cuh -- the Coulomb pass of the pair Poisson solves (Eq. 3) on the
// compile-time N^3 boxes: forward FFT along z, times the Coulomb kernel
// 4 pi / |G|^2 / N (G = 0 dropped), inverse FFT along z.
//
// Geometry: every z line (pencil) belongs to two lanes of one warp (lanes l
// and l + 16), which split its butterflies, so stages need only __syncwarp and
// no block-wide barrier exists.  A warp owns G <= 16 consecutive pencils of
// the plane (G consecutive complex values per z row, 8 G bytes, one bulk copy
// each), so at every step each half-warp touches G adjacent shared-memory
// words (no bank conflicts) and G adjacent global words (full sectors).
// Blocks are one warp.
//
// Per pencil the stages are: forward stages 0 .. S-2 in shared memory; the
// last forward stage, the Coulomb factors and the first inverse stage fused
// in registers (they act on the same butterflies); inverse stages S-2 .. 1 in
// shared memory; inverse stage 0 from shared memory straight to global memory.
// The Coulomb factors come from a table in the spectrum's own layout
// (digit-reversed z position, then the plane's stored slot), read once per
// element; the pass itself never needs to know the plane layout.
#pragma once

#include "fft_core.cuh"
#include "internal.h"
#include "tma.cuh"

namespace ace {
namespace zline_detail {

// Stage of the forward (SGN < 0) or inverse (SGN > 0) transform on one pencil
// held in shared memory with element stride G.
template <int RAD, int SGN, int N, int LB, int G>
__device__ __forceinline__ void pencil_stage(cx<float>* col, const cx<float>* tw, int h) {
    constexpr int M = LB / RAD, NB = N / RAD, TS = N / LB;
#pragma unroll 2
    for (int i = h; i < NB; i += 2) {
        const int beta = i / M, j = i - beta * M;
        butterfly_core<RAD, SGN, float>(col + (beta * LB + j) * G, M * G, tw, TS * j, M > 1 && j > 0);
    }
}

// Last forward stage (blocks of RAD adjacent positions, no twiddles), the
// Coulomb factors, and the first inverse stage on the same RAD positions.
template <int RAD, int N, int G>
__device__ __forceinline__ void pencil_middle(cx<float>* col, const float* krow, int h) {
    constexpr int NB = N / RAD;
    constexpr long long NN = (long long)N * N;
#pragma unroll 2
    for (int beta = h; beta < NB; beta += 2) {
        float k[RAD];
        cx<float> u[RAD];
#pragma unroll
        for (int q = 0; q < RAD; ++q) k[q] = __ldg(krow + (beta * RAD + q) * NN);
#pragma unroll
        for (int q = 0; q < RAD; ++q) u[q] = col[(beta * RAD + q) * G];
        Dft<RAD, -1, float>::run(u);
#pragma unroll
        for (int q = 0; q < RAD; ++q) u[q] = scale(u[q], k[q]);
        Dft<RAD, +1, float>::run(u);
#pragma unroll
        for (int q = 0; q < RAD; ++q) col[(beta * RAD + q) * G] = u[q];
    }
}

// Inverse stage 0 (blocks of the whole line): conjugate twiddles, butterfly,
// and the results in natural order straight to global memory (stride N^2).
template <int RAD, int N, int G>
__device__ __forceinline__ void pencil_last(const cx<float>* col, const cx<float>* tw, cx<float>* out, int h) {
    constexpr int M = N / RAD;
    constexpr long long NN = (long long)N * N;
#pragma unroll 2
    for (int j = h; j < M; j += 2) {
        cx<float> u[RAD];
#pragma unroll
        for (int q = 0; q < RAD; ++q) u[q] = col[(j + q * M) * G];
        if (j > 0) {
#pragma unroll
            for (int q = 1; q < RAD; ++q) {
                cx<float> w = tw[q * j];
                w.im = -w.im;
                u[q] = cmul(u[q], w);
            }
        }
        Dft<RAD, +1, float>::run(u);
#pragma unroll
        for (int s = 0; s < RAD; ++s) out[(j + s * M) * NN] = u[s];
    }
}

// The transforms of one group of G pencils held in buf ([N][G], element
// stride G), by one warp: forward stages, the fused middle with the Coulomb
// factors kern_p0[z N^2 + p], the inverse stages, and the results to
// dst_p0[z N^2 + p] (p = 0 .. G-1, in natural z order).
template <int N, int G, int F0 = 0>
__device__ __forceinline__ void pencils_compute(cx<float>* buf, const cx<float>* tw, const float* kern_p0,
                                                cx<float>* dst_p0, int lane) {
    using PL = CPlan<N, F0>;
    // lanes past the group's pencils (G < 16) skip every step but the syncs
    const int pl = lane & 15, h = lane >> 4;
    const bool on = pl < G;
    cx<float>* col = buf + pl;
    CLoop<0, PL::stages - 1>::run([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        if (on) pencil_stage<PL::radix(s), -1, N, PL::block_len(s), G>(col, tw, h);
        __syncwarp();
    });
    if (on) pencil_middle<PL::radix(PL::stages - 1), N, G>(col, kern_p0 + pl, h);
    __syncwarp();
    CLoop<0, PL::stages - 2>::run([&](auto sc) {
        constexpr int s = PL::stages - 2 - decltype(sc)::value;
        if (on) pencil_stage<PL::radix(s), +1, N, PL::block_len(s), G>(col, tw, h);
        __syncwarp();
    });
    cx<float>* out = dst_p0 + pl;
    if (on) pencil_last<PL::radix(0), N, G>(col, tw, out, h);
}

template <int N, int G, int F0>
__global__ void __launch_bounds__(32) zline_coulomb(PassArgs a) {
    using PL = CPlan<N, F0>;
    static_assert(PL::stages >= 2, "the fused middle needs two stages or more");
    static_assert(G % 2 == 0 && G <= 16 && (N * N) % G == 0, "pencil group");
    constexpr long long NN = (long long)N * N;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    cx<float>* buf = reinterpret_cast<cx<float>*>(smem_raw);  // [N][G]
    cx<float>* tw = buf + N * G;                               // [N]
    const int lane = threadIdx.x;
    const long long p0 = (long long)blockIdx.x * G;
    const int t = blockIdx.y;
    const cx<float>* src = reinterpret_cast<const cx<float>*>(a.src) + t * a.src_tstride + p0;

    if (lane == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, (uint32_t)(N * G * sizeof(cx<float>)));
    }
    __syncwarp();
    for (int z = lane; z < N; z += 32) bulk_load(buf + z * G, src + z * NN, (uint32_t)(G * sizeof(cx<float>)), &bar);
    for (int j = lane; j < N; j += 32) tw[j] = reinterpret_cast<const cx<float>*>(a.twz)[j];
    __syncwarp();
    if (!mbar_wait_bounded(&bar, 0, a.err, 1)) {
        // copies still in flight land in this block's shared memory: give them
        // a second bounded wait before the block leaves
        mbar_wait_bounded(&bar, 0, nullptr, 0);
        return;
    }
    pencils_compute<N, G, F0>(buf, tw, reinterpret_cast<const float*>(a.kern) + p0,
                          reinterpret_cast<cx<float>*>(a.dst) + t * a.dst_tstride + p0, lane);
}

}  // namespace zline_detail

// F0: the first radix of the z axis (0: make_axis_plan's choice)
template <int N, int F0 = 0>
cudaError_t zline_launch(const PassArgs& a, int batch, cudaStream_t st) {
    constexpr int G = zline_group(N);
    auto k = zline_detail::zline_coulomb<N, G, F0>;
    static bool carveout = [&] {
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        cudaGetLastError();
        return true;
    }();
    (void)carveout;
    const size_t smem = (size_t)(N * G + N) * sizeof(cx<float>);
    dim3 grid((unsigned)(N * N / G), (unsigned)batch);
    k<<<grid, 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ace
