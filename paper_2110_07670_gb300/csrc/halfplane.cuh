// halfplane.cuh -- the two plane passes of the pair Poisson solves (Eq. 2-4)
// on a pair of thread blocks (a cluster of two), each holding half a plane.
//
// An N x N complex plane of the 120^3 box takes 115 KB of shared memory, so a
// whole-plane block leaves one block per SM; half a plane (N / 2 rows or
// columns, 58 KB) lets three run.  Block r of the pair owns columns
// [r H, r H + H) of the plane in one layout and rows [r H, r H + H) in the
// other (H = N / 2); between the two axes' transforms the pair trades the
// quarters each needs through distributed shared memory:
//
//   forward  (P1):  pair products for my columns ([N][H]), y transform, trade,
//                   x transform of my rows ([H][N]), rows out to the spectrum
//                   plane (the tile passes' natural layout);
//   inverse  (P3):  my rows of the spectrum plane in ([H][N]), x transform,
//                   trade, y transform of my columns ([N][H]), then the
//                   exchange accumulation W_a += v phi_b ... and the pair
//                   energies (Eq. 2, 4) on my columns.
//
// The trade: after a cluster barrier every thread reads its share of the new
// layout from its own and the peer's tile into registers, a second cluster
// barrier waits until both blocks have read, and the registers go to the new
// layout.  Both blocks of a pair always pass both barriers (no early return
// exists in these kernels).
#pragma once

#include "fft_core.cuh"
#include "internal.h"
#include "tma.cuh"

namespace ace {
namespace half_detail {

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same variable in block `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

template <int N, int F0>
struct HGeo {
    static_assert(N % 8 == 0, "half planes of whole 4-wide vectors");
    static constexpr int H = N / 2;
    static constexpr int NT = 256;
    static constexpr int E = H * N;                    // complex elements per block
    static constexpr int KR = (E + NT - 1) / NT;       // trade registers per thread
    static constexpr size_t smem = (size_t)(E + N) * sizeof(cx<float>);  // tile, twiddles
};

// The trade.  to_rows: from my columns ([N][H], element (y, xl) at y H + xl)
// to my rows ([H][N], (yl, x) at yl N + x); otherwise back.  Block r owns
// columns / rows [r H, r H + H).
template <int N, int F0, bool TO_ROWS>
__device__ __forceinline__ void trade(cx<float>* tile, int r) {
    using G = HGeo<N, F0>;
    constexpr int H = G::H;
    const uint32_t peer = peer_addr(tile, (uint32_t)(r ^ 1));
    cluster_sync();  // both blocks' transforms are done
    float2 v[G::KR];
#pragma unroll
    for (int k = 0; k < G::KR; ++k) {
        const int e = (int)threadIdx.x + k * G::NT;
        if (e < G::E) {
            int src;  // the element's place in its owner's old layout, and the owner
            bool mine;
            if (TO_ROWS) {
                const int yl = e / N, x = e - yl * N, cb = x / H;
                src = (r * H + yl) * H + (x - cb * H);
                mine = cb == r;
            } else {
                const int y = e / H, xl = e - y * H, rb = y / H;
                src = (y - rb * H) * N + r * H + xl;
                mine = rb == r;
            }
            if (mine) {
                const cx<float> c = tile[src];
                v[k] = make_float2(c.re, c.im);
            } else {
                v[k] = ld_cluster(peer + (uint32_t)src * (uint32_t)sizeof(cx<float>));
            }
        }
    }
    cluster_sync();  // both blocks have read what they need from the other
#pragma unroll
    for (int k = 0; k < G::KR; ++k) {
        const int e = (int)threadIdx.x + k * G::NT;
        if (e < G::E) tile[e] = mk(v[k].x, v[k].y);
    }
    __syncthreads();
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void red_add4(float* p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// P1: plane z of transform t (quad q) -> spectrum plane rows [r H, r H + H).
template <int N, int F0>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(HGeo<N, F0>::NT, 3) half_fwd(PassArgs a) {
    using G = HGeo<N, F0>;
    constexpr int H = G::H;
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<float>* tile = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tw = tile + G::E;
    const int r = (int)cluster_rank(), z = blockIdx.x >> 1, t = blockIdx.y;
    const Quad q = a.quads[a.t0 + t];
    const long long plane0 = (long long)z * NN;
    for (int j = threadIdx.x; j < N; j += G::NT) tw[j] = reinterpret_cast<const cx<float>*>(a.twx)[j];
    // pair densities of my columns: rho = phi_a phi_b + i phi_c phi_d
    {
        const float* fl = reinterpret_cast<const float*>(a.fl);
        const float* fr = reinterpret_cast<const float*>(a.fr);
        const bool has2 = q.c >= 0;
        const float* pa = fl + q.a * N3 + plane0 + r * H;
        const float* pb = fr + q.b * N3 + plane0 + r * H;
        const float* pc = fl + (has2 ? q.c : q.a) * N3 + plane0 + r * H;
        const float* pd = fr + (has2 ? q.d : q.b) * N3 + plane0 + r * H;
        for (int g = threadIdx.x; g < N * (H / 4); g += G::NT) {
            const int y = g / (H / 4), x4 = (g - y * (H / 4)) * 4;
            const long long o = (long long)y * N + x4;
            const float4 va = ldg4(pa + o), vb = ldg4(pb + o);
            float4 vc = make_float4(0.f, 0.f, 0.f, 0.f), vd = vc;
            if (has2) {
                vc = ldg4(pc + o);
                vd = ldg4(pd + o);
            }
            cx<float>* dst = tile + y * H + x4;
            dst[0] = mk(va.x * vb.x, vc.x * vd.x);
            dst[1] = mk(va.y * vb.y, vc.y * vd.y);
            dst[2] = mk(va.z * vb.z, vc.z * vd.z);
            dst[3] = mk(va.w * vb.w, vc.w * vd.w);
        }
    }
    __syncthreads();
    static_fft<-1, N, H, H, 1, G::NT, float, F0>(tile, tw);  // y lines: my columns
    trade<N, F0, true>(tile, r);
    static_fft<-1, N, H, 1, N, G::NT, float, F0>(tile, tw);  // x lines: my rows
    // my rows of the spectrum plane, 16 bytes (two elements) per store
    cx<float>* out = reinterpret_cast<cx<float>*>(a.dst) + t * a.dst_tstride + plane0 + (long long)r * H * N;
    for (int e = 2 * threadIdx.x; e < G::E; e += 2 * G::NT)
        *reinterpret_cast<float4*>(out + e) = *reinterpret_cast<const float4*>(tile + e);
}

// P3: spectrum plane z of transform t, my rows in; inverse transforms; the
// exchange accumulation and pair energies on my columns.
template <int N, int F0>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(HGeo<N, F0>::NT, 3) half_inv(PassArgs a) {
    using G = HGeo<N, F0>;
    constexpr int H = G::H;
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * (G::NT / 32)];
    cx<float>* tile = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tw = tile + G::E;
    const int r = (int)cluster_rank(), z = blockIdx.x >> 1, t = blockIdx.y;
    const Quad q = a.quads[a.t0 + t];
    const long long plane0 = (long long)z * NN;
    const cx<float>* in =
        reinterpret_cast<const cx<float>*>(a.src) + t * a.src_tstride + plane0 + (long long)r * H * N;
    for (int e = 2 * threadIdx.x; e < G::E; e += 2 * G::NT) {
        float4 v;
        asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "l"(in + e));
        *reinterpret_cast<float4*>(tile + e) = v;
    }
    for (int j = threadIdx.x; j < N; j += G::NT) tw[j] = reinterpret_cast<const cx<float>*>(a.twx)[j];
    __syncthreads();
    static_fft<+1, N, H, 1, N, G::NT, float, F0>(tile, tw);  // x lines: my rows
    trade<N, F0, false>(tile, r);
    static_fft<+1, N, H, H, 1, G::NT, float, F0>(tile, tw);  // y lines: my columns

    // W_a += v1 phi_b (+ v2 phi_d when both pairs share a), W_b += v1 f_a,
    // W_c += v2 phi_d, W_d += v2 f_c, and the pair energies, on my columns
    float e1 = 0.f, e2 = 0.f;
    {
        const float* fl = reinterpret_cast<const float*>(a.fl);
        const float* fr = reinterpret_cast<const float*>(a.fr);
        float* accl = reinterpret_cast<float*>(a.accl);
        float* accr = reinterpret_cast<float*>(a.accr);
        const bool has2 = q.c >= 0, share = has2 && q.c == q.a, sym = a.symmetric != 0;
        const bool upd_b = sym && q.a != q.b, upd_d = sym && has2 && q.c != q.d;
        const long long col0 = plane0 + r * H;
        const float* la_p = fl + q.a * N3 + col0;
        const float* rb_p = fr + q.b * N3 + col0;
        const float* lc_p = fl + (has2 ? q.c : q.a) * N3 + col0;
        const float* rd_p = fr + (has2 ? q.d : q.b) * N3 + col0;
        float* wa_p = accl + q.a * N3 + col0;
        float* wc_p = accl + (has2 ? q.c : q.a) * N3 + col0;
        float* wb_p = sym ? accr + q.b * N3 + col0 : nullptr;
        float* wd_p = sym ? accr + (has2 ? q.d : q.b) * N3 + col0 : nullptr;
        for (int g = threadIdx.x; g < N * (H / 4); g += G::NT) {
            const int y = g / (H / 4), x4 = (g - y * (H / 4)) * 4;
            const long long o = (long long)y * N + x4;
            const float4 la = ldg4(la_p + o), rb = ldg4(rb_p + o);
            float4 lc = make_float4(0.f, 0.f, 0.f, 0.f), rd = lc;
            if (has2) {
                lc = ldg4(lc_p + o);
                rd = ldg4(rd_p + o);
            }
            const float4 p0 = *reinterpret_cast<const float4*>(tile + y * H + x4);
            const float4 p1 = *reinterpret_cast<const float4*>(tile + y * H + x4 + 2);
            const float4 v1 = make_float4(p0.x, p0.z, p1.x, p1.z);  // real parts: pair 1
            const float4 v2 = make_float4(p0.y, p0.w, p1.y, p1.w);  // imaginary parts: pair 2
            float4 wa = make_float4(v1.x * rb.x, v1.y * rb.y, v1.z * rb.z, v1.w * rb.w);
            e1 += la.x * rb.x * v1.x + la.y * rb.y * v1.y + la.z * rb.z * v1.z + la.w * rb.w * v1.w;
            if (has2) {
                e2 += lc.x * rd.x * v2.x + lc.y * rd.y * v2.y + lc.z * rd.z * v2.z + lc.w * rd.w * v2.w;
                const float4 wc = make_float4(v2.x * rd.x, v2.y * rd.y, v2.z * rd.z, v2.w * rd.w);
                if (share)
                    wa = make_float4(wa.x + wc.x, wa.y + wc.y, wa.z + wc.z, wa.w + wc.w);
                else
                    red_add4(wc_p + o, wc);
                if (upd_d) red_add4(wd_p + o, make_float4(v2.x * lc.x, v2.y * lc.y, v2.z * lc.z, v2.w * lc.w));
            }
            red_add4(wa_p + o, wa);
            if (upd_b) red_add4(wb_p + o, make_float4(v1.x * la.x, v1.y * la.y, v1.z * la.z, v1.w * la.w));
        }
    }
    if (a.e_part != nullptr) {
        const double d1 = warp_sum_ff(e1), d2 = warp_sum_ff(e2);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            red[2 * warp] = d1;
            red[2 * warp + 1] = d2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s1 = 0, s2 = 0;
            for (int w = 0; w < G::NT / 32; ++w) {
                s1 += red[2 * w];
                s2 += red[2 * w + 1];
            }
            double* dst = a.e_part + ((long long)(a.t0 + t) * gridDim.x + blockIdx.x) * 2;
            dst[0] = s1;
            dst[1] = s2;
        }
    }
}

}  // namespace half_detail

// which: 0 = pair product + forward (P1), 1 = inverse + exchange accumulation
// (P3); the grid's x is 2 N (plane z, block r of its pair at 2 z + r)
template <int N, int F0 = 0>
cudaError_t halfplane_launch(int which, const PassArgs& a, int batch, cudaStream_t st) {
    using G = half_detail::HGeo<N, F0>;
    auto k = which == 0 ? half_detail::half_fwd<N, F0> : half_detail::half_inv<N, F0>;
    if (!stream_capturing(st)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(2 * N), (unsigned)batch);
    k<<<grid, G::NT, G::smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ace
