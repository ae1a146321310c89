// plane.cuh -- the two plane passes of the pair Poisson solves (Eq. 2-4) on
// the compile-time N^3 boxes, with thread-owned lines:
//
//   forward  (pair_fwd):   rho = phi_a phi_b + i phi_c phi_d on plane z, 2-D
//                          forward FFT, spectrum plane stored TRANSPOSED;
//   inverse  (inv_accum):  2-D inverse FFT of a transposed spectrum plane,
//                          then W_a += v phi_b, W_b += v phi_a, ... and the
//                          pair energies sum rho v (Eq. 4).
//
// Between the passes (and through the per-pencil Coulomb pass) a spectrum
// plane is stored as [x][y] (x position major, both positions digit-reversed
// after the forward stages).  That lets the pass that works on x lines read
// or write global memory straight from its butterflies with the lanes along
// y (coalesced), while the pass that works on y lines meets the real-space
// functions with the lanes along x (coalesced).
//
// Every line (a y column or an x row of the plane) belongs to two threads,
// thread l and thread N + l (four, up to 3N + l, on the planes of 120^3 and
// up, which leave one block per SM), which split its butterflies; a warp's lanes take
// 32 consecutive lines, so a load of the functions' row segment is one
// 128-byte line, and the two halves of a line meet at block barriers between
// the stages.  The shared tile has an odd row pitch (N + 1), so 16 lanes on
// 16 consecutive rows, or on 16 consecutive columns, hit 16 distinct bank
// pairs.  The accumulation after the inverse runs on 4-wide vectors from
// the shared tile (a final block barrier).  Both axes have two stages (radix R0 with N / R0 butterflies of
// stride N / R0, then radix R1 on adjacent positions).
#pragma once

#include "fft_core.cuh"
#include "internal.h"
#include "tma.cuh"

namespace ace {
namespace plane_detail {

// F0: the first radix of both axes (0: make_axis_plan's choice); TPL: threads
// per line (2, or 4 for the large planes that leave one block per SM)
template <int N, int F0 = 0, int TPL = 2>
struct Geo {
    using PL = CPlan<N, F0>;
    static_assert(PL::stages == 2, "plane passes assume two stages per axis");
    static constexpr int R0 = PL::radix(0), R1 = PL::radix(1);
    static constexpr int M0 = N / R0;  // stage-0 butterflies per line (stride M0)
    static constexpr int B1 = N / R1;  // stage-1 butterflies per line (adjacent)
    static constexpr int P = N + 1;    // shared row pitch, odd
    static constexpr int NT = (TPL * N + 31) / 32 * 32;
    static constexpr size_t smem = (size_t)(N * P + N) * sizeof(cx<float>);
    // resident blocks per SM: 228 KB of shared memory, 1 KB reserved per block
    // (and a little static shared memory)
    static constexpr int kSmemBlocks = 3 * (smem + 1280) <= 228 * 1024 ? 3 : (2 * (smem + 1280) <= 228 * 1024 ? 2 : 1);
    // and no more blocks than leave 72 registers per thread
    static constexpr int kRegBlocks = 65536 / (NT * 72) > 0 ? 65536 / (NT * 72) : 1;
    static constexpr int kMinBlocks = kSmemBlocks < kRegBlocks ? kSmemBlocks : kRegBlocks;
};

// forward stage-0 twiddles on the outputs (DIF), inverse on the inputs (conjugate)
template <int R>
__device__ __forceinline__ void tw_out(cx<float> (&u)[R], const cx<float>* tw, int j) {
    if (j > 0) {
#pragma unroll
        for (int s = 1; s < R; ++s) u[s] = cmul(u[s], tw[s * j]);
    }
}
template <int R>
__device__ __forceinline__ void tw_in_conj(cx<float> (&u)[R], const cx<float>* tw, int j) {
    if (j > 0) {
#pragma unroll
        for (int q = 1; q < R; ++q) {
            cx<float> w = tw[q * j];
            w.im = -w.im;
            u[q] = cmul(u[q], w);
        }
    }
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 mul4(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }
__device__ __forceinline__ float4 fma4(float4 a, float4 b, float4 c) {
    return make_float4(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y), fmaf(a.z, b.z, c.z), fmaf(a.w, b.w, c.w));
}
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ void red_add4(float* p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// 8-byte global -> shared asynchronous copy (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Pull the plane-z slices of transform tt's functions (and accumulators) into L2.
__device__ __forceinline__ void prefetch_planes(const PassArgs& a, const Quad& q, long long off, uint32_t bytes,
                                                long long N3, bool with_w) {
    const float* fl = reinterpret_cast<const float*>(a.fl);
    const float* fr = reinterpret_cast<const float*>(a.fr);
    prefetch_l2(fl + q.a * N3 + off, bytes);
    prefetch_l2(fr + q.b * N3 + off, bytes);
    if (q.c >= 0) {
        if (q.c != q.a) prefetch_l2(fl + q.c * N3 + off, bytes);
        prefetch_l2(fr + q.d * N3 + off, bytes);
    }
    if (with_w) {
        const float* wl = reinterpret_cast<const float*>(a.accl);
        prefetch_l2(wl + q.a * N3 + off, bytes);
        if (q.c >= 0 && q.c != q.a) prefetch_l2(wl + q.c * N3 + off, bytes);
        if (a.symmetric) {
            const float* wr = reinterpret_cast<const float*>(a.accr);
            if (q.b != q.a) prefetch_l2(wr + q.b * N3 + off, bytes);
            if (q.c >= 0 && q.d != q.c) prefetch_l2(wr + q.d * N3 + off, bytes);
        }
    }
}

// Plane z of one transform (quad q): pair product, 2-D forward FFT, and the
// plane stored into spec_t (the transform's spectrum): transposed ([x][y]),
// or with NATURAL in the tile passes' layout (row y, x position p in slot
// plane_swizzle(p, y)), through the shared tile and one more block barrier.
// tw holds the N twiddles in shared memory (visible to the block); the
// block's threads all call this.
template <int N, bool NATURAL = false, int F0 = 0, int TPL = 2>
__device__ __forceinline__ void pair_fwd_plane(const PassArgs& a, const Quad& q, int z, cx<float>* tile,
                                               const cx<float>* tw, cx<float>* spec_t) {
    using G = Geo<N, F0, TPL>;
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    const long long plane0 = (long long)z * NN;
    const int h = (int)threadIdx.x / N, line = (int)threadIdx.x - h * N;
    const bool active = h < TPL;  // threads past TPL N idle
    const bool has2 = q.c >= 0;

    // y lines (thread owns column x): stage 0 straight from the functions
    if (active) {
        const int x = line;
        const float* pa = reinterpret_cast<const float*>(a.fl) + q.a * N3 + plane0 + x;
        const float* pb = reinterpret_cast<const float*>(a.fr) + q.b * N3 + plane0 + x;
        const float* pc = reinterpret_cast<const float*>(a.fl) + (has2 ? q.c : q.a) * N3 + plane0 + x;
        const float* pd = reinterpret_cast<const float*>(a.fr) + (has2 ? q.d : q.b) * N3 + plane0 + x;
        for (int j = h; j < G::M0; j += TPL) {
            cx<float> u[G::R0];
#pragma unroll
            for (int k = 0; k < G::R0; ++k) {
                const long long r = (long long)(j + k * G::M0) * N;
                u[k].re = __ldg(pa + r) * __ldg(pb + r);
                u[k].im = has2 ? __ldg(pc + r) * __ldg(pd + r) : 0.0f;
            }
            Dft<G::R0, -1, float>::run(u);
            tw_out<G::R0>(u, tw, j);
#pragma unroll
            for (int s = 0; s < G::R0; ++s) tile[(j + s * G::M0) * G::P + x] = u[s];
        }
    }
    __syncthreads();
    if (active) {
        const int x = line;
        for (int b = h; b < G::B1; b += TPL) {
            cx<float> u[G::R1];
#pragma unroll
            for (int k = 0; k < G::R1; ++k) u[k] = tile[(b * G::R1 + k) * G::P + x];
            Dft<G::R1, -1, float>::run(u);
#pragma unroll
            for (int s = 0; s < G::R1; ++s) tile[(b * G::R1 + s) * G::P + x] = u[s];
        }
    }
    __syncthreads();

    // x lines (thread owns row y): stage 0 in shared memory, stage 1 to the
    // transposed spectrum plane
    if (active) {
        cx<float>* row = tile + line * G::P;
        for (int j = h; j < G::M0; j += TPL) {
            cx<float> u[G::R0];
#pragma unroll
            for (int k = 0; k < G::R0; ++k) u[k] = row[j + k * G::M0];
            Dft<G::R0, -1, float>::run(u);
            tw_out<G::R0>(u, tw, j);
#pragma unroll
            for (int s = 0; s < G::R0; ++s) row[j + s * G::M0] = u[s];
        }
    }
    __syncthreads();
    if (active) {
        cx<float>* row = tile + line * G::P;
        cx<float>* out = spec_t + plane0 + line;
        for (int b = h; b < G::B1; b += TPL) {
            cx<float> u[G::R1];
#pragma unroll
            for (int k = 0; k < G::R1; ++k) u[k] = row[b * G::R1 + k];
            Dft<G::R1, -1, float>::run(u);
            if constexpr (NATURAL) {
#pragma unroll
                for (int s = 0; s < G::R1; ++s) row[b * G::R1 + s] = u[s];
            } else {
#pragma unroll
                for (int s = 0; s < G::R1; ++s) out[(long long)(b * G::R1 + s) * N] = u[s];
            }
        }
    }
    if constexpr (NATURAL) {
        // rows out with the lanes along x: 32 consecutive positions per warp,
        // permuted within 16-blocks by the slot swizzle, stay coalesced
        __syncthreads();
        cx<float>* out = spec_t + plane0;
        for (int e = threadIdx.x; e < N * N; e += G::NT) {
            const int y = e / N, x = e - y * N;
            out[y * N + (cube_swizzle(N) ? plane_swizzle(x, y, N) : x)] = tile[y * G::P + x];
        }
    }
}

template <int N, bool NATURAL, int F0, int TPL>
__global__ void __launch_bounds__(Geo<N, F0, TPL>::NT, Geo<N, F0, TPL>::kMinBlocks) pair_fwd(PassArgs a) {
    using G = Geo<N, F0, TPL>;
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<float>* tile = reinterpret_cast<cx<float>*>(smem_raw);  // (y, x) at y * P + x
    cx<float>* tw = tile + N * G::P;
    const int z = blockIdx.x, t = blockIdx.y;
    const Quad q = a.quads[a.t0 + t];
    const long long plane0 = (long long)z * NN;
    for (int j = threadIdx.x; j < N; j += G::NT) tw[j] = reinterpret_cast<const cx<float>*>(a.twx)[j];
    if (threadIdx.x == 32 && a.lookahead > 0 && t + a.lookahead < (int)gridDim.y && (NN * 4) % 16 == 0)
        prefetch_planes(a, a.quads[a.t0 + t + a.lookahead], plane0, (uint32_t)(NN * 4), N3, false);
    __syncthreads();
    pair_fwd_plane<N, NATURAL, F0, TPL>(a, q, z, tile, tw, reinterpret_cast<cx<float>*>(a.dst) + t * a.dst_tstride);
}

// Inputs of the inverse pass: thread (row y, half h) needs the transposed
// plane's x positions of its first butterflies in its row of the tile.
// Asynchronous 8-byte copies (the standalone kernel: all in flight at once,
// completed by cp_async_wait_all) ...
template <int N, int F0 = 0, int TPL = 2>
__device__ __forceinline__ void inv_issue_copies(const cx<float>* plane_in, cx<float>* tile) {
    using G = Geo<N, F0, TPL>;
    const int h = (int)threadIdx.x / N, line = (int)threadIdx.x - h * N;
    if (h < TPL) {
        const cx<float>* in = plane_in + line;
        cx<float>* row = tile + line * G::P;
        for (int b = h; b < G::B1; b += TPL)
#pragma unroll
            for (int k = 0; k < G::R1; ++k) cp_async8(row + b * G::R1 + k, in + (long long)(b * G::R1 + k) * N);
    }
    cp_async_commit();
}

// ... or loads that bypass L1 (ld.global.cg), for spectra written by other
// blocks of the same kernel.
__device__ __forceinline__ cx<float> ld_cg2(const cx<float>* p) {
    float2 v;
    asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return mk(v.x, v.y);
}
template <int N, int F0 = 0, int TPL = 2>
__device__ __forceinline__ void inv_load_cg(const cx<float>* plane_in, cx<float>* tile) {
    using G = Geo<N, F0, TPL>;
    const int h = (int)threadIdx.x / N, line = (int)threadIdx.x - h * N;
    if (h < TPL) {
        const cx<float>* in = plane_in + line;
        cx<float>* row = tile + line * G::P;
        for (int b = h; b < G::B1; b += TPL) {
            cx<float> u[G::R1];
#pragma unroll
            for (int k = 0; k < G::R1; ++k) u[k] = ld_cg2(in + (long long)(b * G::R1 + k) * N);
#pragma unroll
            for (int k = 0; k < G::R1; ++k) row[b * G::R1 + k] = u[k];
        }
    }
}

// Plane z of one transform (quad q), its inputs already in the tile (each
// thread's own): 2-D inverse FFT, then W_a += v phi_b, W_b += v phi_a, ...
// (Eq. 2) and the pair-energy partials (Eq. 4) into e_dst[2] (may be null).
// red: 2 * NT / 32 doubles of shared memory.  Every thread of the block calls it.
template <int N, int F0 = 0, int TPL = 2>
__device__ __forceinline__ void inv_accum_plane(const PassArgs& a, const Quad& q, int z, cx<float>* tile,
                                                const cx<float>* tw, double* red, double* e_dst) {
    using G = Geo<N, F0, TPL>;
    static_assert(N % 8 == 0, "the vector epilogue tiles planes by 4 rows x 16 (or 8) columns");
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    const long long plane0 = (long long)z * NN;
    const int h = (int)threadIdx.x / N, line = (int)threadIdx.x - h * N;
    const bool active = h < TPL;  // threads past TPL N idle
    // x lines (thread owns row y): both inverse stages in shared memory
    if (active) {
        cx<float>* row = tile + line * G::P;
        for (int b = h; b < G::B1; b += TPL) {
            cx<float> u[G::R1];
#pragma unroll
            for (int k = 0; k < G::R1; ++k) u[k] = row[b * G::R1 + k];
            Dft<G::R1, +1, float>::run(u);
#pragma unroll
            for (int s = 0; s < G::R1; ++s) row[b * G::R1 + s] = u[s];
        }
    }
    __syncthreads();
    if (active) {
        cx<float>* row = tile + line * G::P;
        for (int j = h; j < G::M0; j += TPL) {
            cx<float> u[G::R0];
#pragma unroll
            for (int k = 0; k < G::R0; ++k) u[k] = row[j + k * G::M0];
            tw_in_conj<G::R0>(u, tw, j);
            Dft<G::R0, +1, float>::run(u);
#pragma unroll
            for (int s = 0; s < G::R0; ++s) row[j + s * G::M0] = u[s];
        }
    }
    __syncthreads();

    // y lines (thread owns column x): both inverse stages in shared memory
    if (active) {
        const int x = line;
        for (int b = h; b < G::B1; b += TPL) {
            cx<float> u[G::R1];
#pragma unroll
            for (int k = 0; k < G::R1; ++k) u[k] = tile[(b * G::R1 + k) * G::P + x];
            Dft<G::R1, +1, float>::run(u);
#pragma unroll
            for (int s = 0; s < G::R1; ++s) tile[(b * G::R1 + s) * G::P + x] = u[s];
        }
    }
    __syncthreads();
    if (active) {
        const int x = line;
        for (int j = h; j < G::M0; j += TPL) {
            cx<float> u[G::R0];
#pragma unroll
            for (int k = 0; k < G::R0; ++k) u[k] = tile[(j + k * G::M0) * G::P + x];
            tw_in_conj<G::R0>(u, tw, j);
            Dft<G::R0, +1, float>::run(u);
#pragma unroll
            for (int s = 0; s < G::R0; ++s) tile[(j + s * G::M0) * G::P + x] = u[s];
        }
    }
    __syncthreads();

    // Exchange accumulation (Eq. 2) and pair energies (Eq. 4) in 4-wide
    // vectors: a half-warp takes 4 rows x 16 columns, lane (r, c) the four
    // columns 4c .. 4c + 3 of row r; with the pitch P = 1 (mod 16) its 16
    // lanes read 16 distinct bank pairs.  (N % 16 != 0: a quarter-warp takes
    // 4 rows x 8 columns, and tasks past the plane's are skipped.)
    float e1 = 0.0f, e2 = 0.0f;
    {
        const bool has2 = q.c >= 0, share = has2 && q.c == q.a, sym = a.symmetric != 0;
        const bool upd_b = sym && q.a != q.b, upd_d = sym && has2 && q.c != q.d;
        const float* la_p = reinterpret_cast<const float*>(a.fl) + q.a * N3 + plane0;
        const float* rb_p = reinterpret_cast<const float*>(a.fr) + q.b * N3 + plane0;
        const float* lc_p = reinterpret_cast<const float*>(a.fl) + (has2 ? q.c : q.a) * N3 + plane0;
        const float* rd_p = reinterpret_cast<const float*>(a.fr) + (has2 ? q.d : q.b) * N3 + plane0;
        float* wa_p = reinterpret_cast<float*>(a.accl) + q.a * N3 + plane0;
        float* wc_p = reinterpret_cast<float*>(a.accl) + (has2 ? q.c : q.a) * N3 + plane0;
        float* wb_p = sym ? reinterpret_cast<float*>(a.accr) + q.b * N3 + plane0 : nullptr;
        float* wd_p = sym ? reinterpret_cast<float*>(a.accr) + (has2 ? q.d : q.b) * N3 + plane0 : nullptr;
        constexpr int TW = N % 16 == 0 ? 16 : 8;  // columns per task, TW lanes (4 rows x TW / 4 vectors)
        const int hw = threadIdx.x / TW, l16 = threadIdx.x % TW;
        const int rr = l16 & 3, cc = l16 >> 2;
        // N^2 / (4 TW) tasks over NT / TW lane groups, taken U at a time with
        // every load of the U tasks issued before the first update
        constexpr int HW = G::NT / TW, NTASK = (N / 4) * (N / TW);
        constexpr int PER = (NTASK + HW - 1) / HW, U = PER % 2 == 0 ? 2 : 1;
        constexpr bool EVEN = NTASK % HW == 0;
        for (int k0 = 0; k0 < PER; k0 += U) {
            float4 la[U], rb[U], lc[U], rd[U];
            long long rof[U];
            int sof[U];
            bool on[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int task = hw + (k0 + u) * HW;
                on[u] = EVEN || task < NTASK;
                if (!on[u]) continue;
                const int y = (task / (N / TW)) * 4 + rr, x = (task % (N / TW)) * TW + 4 * cc;
                rof[u] = (long long)y * N + x;
                sof[u] = y * G::P + x;
                la[u] = ldg4(la_p + rof[u]);
                rb[u] = ldg4(rb_p + rof[u]);
                if (has2) {
                    lc[u] = ldg4(lc_p + rof[u]);
                    rd[u] = ldg4(rd_p + rof[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!on[u]) continue;
                const cx<float>* src = tile + sof[u];
                const cx<float> v[4] = {src[0], src[1], src[2], src[3]};
                const float4 v1 = make_float4(v[0].re, v[1].re, v[2].re, v[3].re);
                const float4 v2 = make_float4(v[0].im, v[1].im, v[2].im, v[3].im);
                const long long r = rof[u];
                float4 wa = mul4(v1, rb[u]);
                e1 += dot4(mul4(la[u], rb[u]), v1);
                if (has2) {
                    e2 += dot4(mul4(lc[u], rd[u]), v2);
                    if (share)
                        wa = fma4(v2, rd[u], wa);
                    else
                        red_add4(wc_p + r, mul4(v2, rd[u]));
                    if (upd_d) red_add4(wd_p + r, mul4(v2, lc[u]));
                }
                red_add4(wa_p + r, wa);
                if (upd_b) red_add4(wb_p + r, mul4(v1, la[u]));
            }
        }
    }
    if (e_dst != nullptr) {
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
            e_dst[0] = s1;
            e_dst[1] = s2;
        }
    }
}

template <int N, int F0, int TPL>
__global__ void __launch_bounds__(Geo<N, F0, TPL>::NT, Geo<N, F0, TPL>::kMinBlocks) inv_accum(PassArgs a) {
    using G = Geo<N, F0, TPL>;
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * (G::NT / 32)];
    cx<float>* tile = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tw = tile + N * G::P;
    const int z = blockIdx.x, t = blockIdx.y;
    const long long plane0 = (long long)z * NN;
    inv_issue_copies<N, F0, TPL>(reinterpret_cast<const cx<float>*>(a.src) + t * a.src_tstride + plane0, tile);
    const Quad q = a.quads[a.t0 + t];
    for (int j = threadIdx.x; j < N; j += G::NT) tw[j] = reinterpret_cast<const cx<float>*>(a.twx)[j];
    // the accumulation reads up to four function planes and updates up to four
    // accumulator planes at the end: start pulling them into L2 now
    if (threadIdx.x == 32 && (NN * 4) % 16 == 0) prefetch_planes(a, q, plane0, (uint32_t)(NN * 4), N3, true);
    cp_async_wait_all();
    __syncthreads();
    inv_accum_plane<N, F0, TPL>(a, q, z, tile, tw, red,
                       a.e_part != nullptr ? a.e_part + ((long long)(a.t0 + t) * gridDim.x + z) * 2 : nullptr);
}

template <typename K>
cudaError_t launch_plane(K k, size_t smem, int n, int nt, const PassArgs& a, int batch, cudaStream_t st) {
    if (smem > 48 * 1024 && !stream_capturing(st)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)n, (unsigned)batch);
    k<<<grid, nt, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace plane_detail

// which: 0 = pair product + forward plane FFT (transposed planes out),
// 1 = inverse plane FFT + accumulation, 2 = the forward pass with the tile
// passes' plane layout out (the hybrid variant)
template <int N, int F0 = 0>
cudaError_t tplane_launch(int which, const PassArgs& a, int batch, cudaStream_t st) {
    constexpr int TPL = N >= 120 ? 4 : 2;  // one plane block per SM from 120^3 up: more warps per line (at 96^3 two
                                           // blocks of four threads per line ran P1 4% slower than three of two)
    using G = plane_detail::Geo<N, F0, TPL>;
    if (which == 2)
        return plane_detail::launch_plane(plane_detail::pair_fwd<N, true, F0, TPL>, G::smem, N, G::NT, a, batch, st);
    if constexpr (N % 8 != 0) {
        return cudaErrorInvalidValue;  // transposed planes: n % 8 == 0 only
    } else {
        if (which == 0)
            return plane_detail::launch_plane(plane_detail::pair_fwd<N, false, F0, TPL>, G::smem, N, G::NT, a, batch, st);
        return plane_detail::launch_plane(plane_detail::inv_accum<N, F0, TPL>, G::smem, N, G::NT, a, batch, st);
    }
}

}  // namespace ace
