// pass_kernel.cuh -- the FFT pass kernel of the pair Poisson solves.
//
// A 3D transform of an n0 x n1 x n2 box is done in passes; each thread block
// owns one tile of one transform in shared memory, transforms it along one or
// more axes with the in-place stages of fft_core.cuh, and hands it to an
// epilogue.  The prologues and epilogues fuse the exchange work of
// arXiv:2110.07670 Section 2.1 into the first and last passes:
//
//   pair density (Eq. 3)       rho = f_a phi_b, two pairs packed as re + i im
//   Coulomb solve (Eq. 3)      v(G) = 4 pi / |G|^2 rho(G) / N, G = 0 dropped,
//                              applied between the forward and inverse z axis
//   exchange (Eq. 2)           W_a += v phi_b, W_b += v f_a (a != b)
//   pair energy (Eq. 4)        e_ab = sum_r rho v  (times Omega / N later)
//
// so pair densities and pair potentials never travel through global memory
// between the passes; only the half-transformed spectrum does.  Spectrum
// tiles move with bulk asynchronous copies (TMA) completing on an mbarrier;
// real-space functions move as 16-byte vectors, W updates as vector atomics.
// The kernel is written once over a tile geometry: DynShape (runtime sizes,
// any grid) or CubeShape (compile-time N^3 box and tile).
#pragma once

#include "internal.h"
#include "tma.cuh"

namespace ace {
namespace pass_detail {

__device__ __forceinline__ int fold_index(int i, int n) { return i < n - n / 2 ? i : i - n; }

// 4 consecutive reals as one 16-byte (float) or two 16-byte (double) vectors
template <typename R>
struct V4 {
    R x, y, z, w;
};

template <typename R>
__device__ __forceinline__ V4<R> ld4(const R* p) {
    if constexpr (sizeof(R) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        return V4<R>{v.x, v.y, v.z, v.w};
    } else {
        const double2 u = __ldg(reinterpret_cast<const double2*>(p));
        const double2 v = __ldg(reinterpret_cast<const double2*>(p) + 1);
        return V4<R>{u.x, u.y, v.x, v.y};
    }
}

template <typename R>
__device__ __forceinline__ void st4(R* p, V4<R> v) {
    if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
        reinterpret_cast<double2*>(p)[1] = make_double2(v.z, v.w);
    }
}

template <typename R>
__device__ __forceinline__ void red4(R* p, V4<R> v) {
    if constexpr (sizeof(R) == 4) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                     "f"(v.w)
                     : "memory");
    } else {
        atomicAdd(p, v.x);
        atomicAdd(p + 1, v.y);
        atomicAdd(p + 2, v.z);
        atomicAdd(p + 3, v.w);
    }
}

template <typename R>
__device__ __forceinline__ V4<R> mul4(V4<R> a, V4<R> b) {
    return V4<R>{a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w};
}
template <typename R>
__device__ __forceinline__ V4<R> fma4(V4<R> a, V4<R> b, V4<R> c) {
    return V4<R>{a.x * b.x + c.x, a.y * b.y + c.y, a.z * b.z + c.z, a.w * b.w + c.w};
}
template <typename R>
__device__ __forceinline__ R dot4(V4<R> a, V4<R> b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// Runs of a tile in global memory: rows of tx elements, merged into longer
// runs when the tile spans whole rows or planes of the box.
struct Chunks {
    int count, len;  // number of runs, elements per run
};
template <typename Shape>
__device__ __forceinline__ Chunks tile_chunks(const Shape& a) {
    if (a.tx == a.n2 && a.ty == a.n1) return Chunks{a.tz, a.n1 * a.n2};
    if (a.tx == a.n2) return Chunks{a.tz, a.ty * a.n2};
    return Chunks{a.tz * a.ty, a.tx};
}
// global element offset (within the transform) and tile offset of run k
template <typename Shape>
__device__ __forceinline__ void chunk_at(const Shape& a, int k, int z0, int y0, int x0, long long& g, int& s) {
    if (a.tx == a.n2) {
        g = ((long long)(z0 + k) * a.n1 + y0) * a.n2;
        s = k * a.ty * a.tx;
    } else {
        const int ez = k / a.ty, ey = k - ez * a.ty;
        g = ((long long)(z0 + ez) * a.n1 + (y0 + ey)) * a.n2 + x0;
        s = k * a.tx;
    }
}


// Runtime tile geometry (any grid) ...
struct DynShape {
    static constexpr bool kCube = false;
    static constexpr int kMaxThreads = 512;
    static constexpr int kMinBlocks = 1;
    int n0, n1, n2, tz, ty, tx, axes;
    __device__ explicit DynShape(const PassArgs& a)
        : n0(a.n0), n1(a.n1), n2(a.n2), tz(a.tz), ty(a.ty), tx(a.tx), axes(a.axes) {}
    __device__ int nt() const { return blockDim.x; }
    __device__ static int slot(int e) { return e; }             // tile slot of tile element e
    __device__ static int xpos(int s, int) { return s; }        // x position held in global x slot s
    template <int SGN, typename R>
    __device__ void fft_x(cx<R>* t, const cx<R>* tw, const PassArgs& a) const {
        block_fft<SGN, R>(t, Lines{tx, tz * ty, 1, tx}, a.px, tw);
    }
    template <int SGN, typename R>
    __device__ void fft_y(cx<R>* t, const cx<R>* tw, const PassArgs& a) const {
        block_fft<SGN, R>(t, Lines{ty, tx, tx, 1}, a.py, tw);
    }
    template <int SGN, typename R>
    __device__ void fft_z(cx<R>* t, const cx<R>* tw, const PassArgs& a) const {
        block_fft<SGN, R>(t, Lines{tz, tx * ty, tx * ty, 1}, a.pz, tw);
    }
};

// Stages along the x lines of a swizzled N x N plane (row stride N): the same
// butterflies as static_stage, with each element addressed through
// plane_swizzle so that neither the strided first stage nor the contiguous last
// stage (each butterfly on RAD adjacent positions) collides in the banks.
template <int RAD, int SGN, typename R>
__device__ __forceinline__ void butterfly_at(cx<R>* row, const int (&idx)[RAD], const cx<R>* tw, int tstep,
                                             bool tw_on) {
    cx<R> u[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) u[q] = row[idx[q]];
    if (SGN > 0 && tw_on) {
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
            cx<R> w = tw[q * tstep];
            w.im = -w.im;
            u[q] = cmul(u[q], w);
        }
    }
    Dft<RAD, SGN, R>::run(u);
    if (SGN < 0 && tw_on) {
#pragma unroll
        for (int s = 1; s < RAD; ++s) u[s] = cmul(u[s], tw[s * tstep]);
    }
#pragma unroll
    for (int s = 0; s < RAD; ++s) row[idx[s]] = u[s];
}

// The same butterfly with its twiddles already in registers (w[q] for q > 0,
// conjugated for SGN > 0).
template <int RAD, int SGN, typename R>
__device__ __forceinline__ void butterfly_at_w(cx<R>* row, const int (&idx)[RAD], const cx<R> (&w)[RAD], bool tw_on) {
    cx<R> u[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) u[q] = row[idx[q]];
    if (SGN > 0 && tw_on) {
#pragma unroll
        for (int q = 1; q < RAD; ++q) u[q] = cmul(u[q], w[q]);
    }
    Dft<RAD, SGN, R>::run(u);
    if (SGN < 0 && tw_on) {
#pragma unroll
        for (int s = 1; s < RAD; ++s) u[s] = cmul(u[s], w[s]);
    }
#pragma unroll
    for (int s = 0; s < RAD; ++s) row[idx[s]] = u[s];
}

template <int RAD, int SGN, int N, int LB, int NT, typename R>
__device__ __forceinline__ void static_stage_rows_swizzled(cx<R>* buf, const cx<R>* tw) {
    constexpr int M = LB / RAD, NB = N / RAD, TOTAL = NB * N, TS = N / LB;
    if constexpr (M > 1 && NT % NB == 0) {
        // every butterfly of this thread has the same j (NT is a multiple of
        // the butterflies per row): its twiddles are read once
        const int i = (int)threadIdx.x % NB, j = i % M, beta = i / M;
        cx<R> w[RAD];
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
            w[q] = tw[q * TS * j];
            if (SGN > 0) w[q].im = -w[q].im;
        }
        w[0] = mk(R(1), R(0));
        const int p0 = beta * LB + j;
        for (int line = (int)threadIdx.x / NB; line < N; line += NT / NB) {
            int idx[RAD];
#pragma unroll
            for (int q = 0; q < RAD; ++q) idx[q] = plane_swizzle(p0 + q * M, line, N);
            butterfly_at_w<RAD, SGN, R>(buf + line * N, idx, w, j > 0);
        }
        __syncthreads();
        return;
    }
    for (int b = threadIdx.x; b < TOTAL; b += NT) {
        const int line = b / NB, i = b - line * NB;
        const int beta = i / M, j = i - beta * M;
        const int p0 = beta * LB + j;
        int idx[RAD];
#pragma unroll
        for (int q = 0; q < RAD; ++q) idx[q] = plane_swizzle(p0 + q * M, line, N);
        butterfly_at<RAD, SGN, R>(buf + line * N, idx, tw, TS * j, M > 1 && j > 0);
    }
    __syncthreads();
}

// y lines of the same swizzled plane: line p holds x position p of every row,
// which sits in slot plane_swizzle(p, y) of row y.
template <int RAD, int SGN, int N, int LB, int NT, typename R>
__device__ __forceinline__ void static_stage_cols_swizzled(cx<R>* buf, const cx<R>* tw) {
    constexpr int M = LB / RAD, NB = N / RAD, TOTAL = NB * N, TS = N / LB;
    for (int b = threadIdx.x; b < TOTAL; b += NT) {
        const int i = b / N, p = b - i * N;
        const int beta = i / M, j = i - beta * M;
        const int y0 = beta * LB + j;
        int idx[RAD];
#pragma unroll
        for (int q = 0; q < RAD; ++q) idx[q] = (y0 + q * M) * N + plane_swizzle(p, y0 + q * M, N);
        butterfly_at<RAD, SGN, R>(buf, idx, tw, TS * j, M > 1 && j > 0);
    }
    __syncthreads();
}

template <int SGN, int N, int NT, typename R, int R0 = 0>
__device__ __forceinline__ void static_fft_cols_swizzled(cx<R>* buf, const cx<R>* tw) {
    using PL = CPlan<N, R0>;
    CLoop<0, PL::stages>::run([&](auto sc) {
        constexpr int s = SGN < 0 ? decltype(sc)::value : PL::stages - 1 - decltype(sc)::value;
        static_stage_cols_swizzled<PL::radix(s), SGN, N, PL::block_len(s), NT, R>(buf, tw);
    });
}

template <int SGN, int N, int NT, typename R, int R0 = 0>
__device__ __forceinline__ void static_fft_rows_swizzled(cx<R>* buf, const cx<R>* tw) {
    using PL = CPlan<N, R0>;
    CLoop<0, PL::stages>::run([&](auto sc) {
        constexpr int s = SGN < 0 ? decltype(sc)::value : PL::stages - 1 - decltype(sc)::value;
        static_stage_rows_swizzled<PL::radix(s), SGN, N, PL::block_len(s), NT, R>(buf, tw);
    });
}

// ... and compile-time geometry of an N^3 box with NT threads per block: every
// index division becomes a multiply-shift and every stage loop a fixed count.
// R0: the first radix of every axis (0: make_axis_plan's choice).
template <int N, int TZ, int TY, int TX, int NT, int R0 = 0>
struct CubeShape {
    static constexpr bool kCube = true;
    static constexpr int kMaxThreads = NT;
    // two resident plane blocks where two N x N complex tiles fit in shared
    // memory (N <= 108); otherwise one, with the whole register file for it
    static constexpr bool kPlane = TZ == 1 && TY == N && TX == N;
    static constexpr int kMinBlocks = !kPlane ? 1 : (3 * (N * N * 8 + 2 * N * 8 + 1280) <= 228 * 1024 && NT <= 256) ? 3
                                                  : (2 * (N * N * 8 + 4096) <= 227 * 1024 ? 2 : 1);
    static constexpr int n0 = N, n1 = N, n2 = N, tz = TZ, ty = TY, tx = TX;
    static constexpr int axes = (TZ == 1 && TY == N && TX == N) ? 3 : (TZ == N ? 4 : (TZ == 1 && TX == N ? 1 : 2));
    // Plane tiles of N % 16 == 0 boxes are stored (in shared and global memory)
    // with x position p of row y in slot swizzle_x(p, y); see plane_swizzle.
    static constexpr bool kSwzLayout = cube_swizzle(N);
    static constexpr bool kSwzTile = kSwzLayout && TZ == 1 && TY == N && TX == N;
    __device__ explicit CubeShape(const PassArgs&) {}
    __device__ static constexpr int nt() { return NT; }
    __device__ static int slot(int e) {
        if constexpr (kSwzTile) {
            const int row = e / N, col = e - row * N;
            return row * N + plane_swizzle(col, row, N);
        } else {
            return e;
        }
    }
    __device__ static int xpos(int s, int y) {
        if constexpr (kSwzLayout) return plane_swizzle(s, y, N);
        else return s;
    }
    template <int SGN, typename R>
    __device__ void fft_x(cx<R>* t, const cx<R>* tw, const PassArgs&) const {
        if constexpr (kSwzTile)
            static_fft_rows_swizzled<SGN, N, NT, R, R0>(t, tw);
        else
            static_fft<SGN, N, TZ * TY, 1, TX, NT, R, R0>(t, tw);
    }
    template <int SGN, typename R>
    __device__ void fft_y(cx<R>* t, const cx<R>* tw, const PassArgs&) const {
        if constexpr (kSwzTile)
            static_fft_cols_swizzled<SGN, N, NT, R, R0>(t, tw);
        else
            static_fft<SGN, N, TX, TX, 1, NT, R, R0>(t, tw);
    }
    template <int SGN, typename R>
    __device__ void fft_z(cx<R>* t, const cx<R>* tw, const PassArgs&) const {
        static_fft<SGN, N, TY * TX, TY * TX, 1, NT, R, R0>(t, tw);
    }
};

// The tile's four consecutive elements e .. e + 3 (e a multiple of 4 inside one
// row).  Single-precision compile-time tiles read them as two 16-byte shared
// loads: the plane swizzle keeps an aligned group of four x positions in one
// aligned group of four slots, element i in slot i ^ c with c the low two bits
// of the row's swizzle word: one load takes the slot pair holding elements 0
// and 1, the other the pair holding 2 and 3, and a swap inside each pair
// undoes c's low bit.  (Four 8-byte loads at a 32-byte lane stride conflicted
// 8-way in the banks.)
template <typename Shape, typename R>
__device__ __forceinline__ void tile_load4(const Shape& S, const cx<R>* tile, int e, cx<R> (&v)[4]) {
    if constexpr (sizeof(R) == 4 && Shape::kCube) {
        int base = e, c = 0, first = 0;
        if constexpr (Shape::kSwzTile) {
            const int row = e / Shape::n2, col = e - row * Shape::n2;
            const int k = (((col >> 4) + plane_swizzle_rot(Shape::n2) * row) & 7) | ((row & 1) << 3);
            base = row * Shape::n2 + (col ^ (k & 12));
            c = k & 3;
            first = (col >> 4) & 1;
        }
        // the slot pair holding elements 0 and 1 is h; lanes of neighbouring
        // 16-element blocks load their two pairs in opposite orders, so the 8
        // lanes of a quarter-warp (two blocks) cover all 32 banks per load
        const int h = (c >> 1) & 1;
        const float4 qa = *reinterpret_cast<const float4*>(tile + base + 2 * first);
        const float4 qb = *reinterpret_cast<const float4*>(tile + base + 2 * (first ^ 1));
        const float4 q0 = first == h ? qa : qb;
        const float4 q1 = first == h ? qb : qa;
        const bool sw = (c & 1) != 0;
        v[0] = sw ? mk(q0.z, q0.w) : mk(q0.x, q0.y);
        v[1] = sw ? mk(q0.x, q0.y) : mk(q0.z, q0.w);
        v[2] = sw ? mk(q1.z, q1.w) : mk(q1.x, q1.y);
        v[3] = sw ? mk(q1.x, q1.y) : mk(q1.z, q1.w);
    } else {
        v[0] = tile[S.slot(e)];
        v[1] = tile[S.slot(e + 1)];
        v[2] = tile[S.slot(e + 2)];
        v[3] = tile[S.slot(e + 3)];
    }
}

template <typename Shape, typename R, int PRO, int EPI, int MID, int SGN>
__global__ void __launch_bounds__(Shape::kMaxThreads, Shape::kMinBlocks) tile_pass(PassArgs a) {
    const Shape S(a);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ double red[2 * (Shape::kMaxThreads / 32)];  // a pair of energy partials per warp
    const int tile_elems = S.tz * S.ty * S.tx;
    cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* twx = tile + tile_elems;
    cx<R>* twy = twx + ((S.axes & 1) ? S.n2 : 0);
    cx<R>* twz = twy + ((S.axes & 2) ? S.n1 : 0);
    // Coulomb: G-vector component of every position along each axis
    // (gt[3 j + c] axis 0, then axis 1, then axis 2; positions hold digit-reversed frequencies)
    R* gt = reinterpret_cast<R*>(twz + ((S.axes & 4) ? S.n0 : 0));

    const int t = blockIdx.y;
    const int tiles_x = S.n2 / S.tx, tiles_y = S.n1 / S.ty;
    const int tile_id = blockIdx.x;
    const int bx = tile_id % tiles_x, by = (tile_id / tiles_x) % tiles_y, bz = tile_id / (tiles_x * tiles_y);
    const int z0 = bz * S.tz, y0 = by * S.ty, x0 = bx * S.tx;
    const long long N = (long long)S.n0 * S.n1 * S.n2;
    const int txy = S.tx * S.ty;

    // ---- spectrum tile: bulk asynchronous load, started before anything else
    const bool bulk_in = PRO == PRO_LOAD && a.bulk;
    if (bulk_in) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const Chunks ch = tile_chunks(S);
            const cx<R>* src = reinterpret_cast<const cx<R>*>(a.src) + (long long)t * a.src_tstride;
            if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(tile_elems * sizeof(cx<R>)));
            __syncwarp();
            for (int k = threadIdx.x; k < ch.count; k += 32) {
                long long g;
                int s;
                chunk_at(S, k, z0, y0, x0, g, s);
                bulk_load(tile + s, src + g, (uint32_t)(ch.len * sizeof(cx<R>)), &bar);
            }
        }
    }

    if (MID == MID_COULOMB) {
        const int nsum = S.n0 + S.n1 + S.n2;
        for (int j = threadIdx.x; j < nsum; j += S.nt()) {
            const int ax = j < S.n0 ? 0 : (j < S.n0 + S.n1 ? 1 : 2);
            const int jj = j - (ax == 0 ? 0 : (ax == 1 ? S.n0 : S.n0 + S.n1));
            const int n = ax == 0 ? S.n0 : (ax == 1 ? S.n1 : S.n2);
            const R h = R(fold_index(a.freq[ax][jj], n));
            gt[3 * j] = h * R(a.b[3 * ax]);
            gt[3 * j + 1] = h * R(a.b[3 * ax + 1]);
            gt[3 * j + 2] = h * R(a.b[3 * ax + 2]);
        }
    }
    if (S.axes & 1)
        for (int j = threadIdx.x; j < S.n2; j += S.nt()) twx[j] = reinterpret_cast<const cx<R>*>(a.twx)[j];
    if (S.axes & 2)
        for (int j = threadIdx.x; j < S.n1; j += S.nt()) twy[j] = reinterpret_cast<const cx<R>*>(a.twy)[j];
    if (S.axes & 4)
        for (int j = threadIdx.x; j < S.n0; j += S.nt()) twz[j] = reinterpret_cast<const cx<R>*>(a.twz)[j];

    Quad q = {0, 0, -1, 0};
    if (PRO != PRO_LOAD || EPI != EPI_STORE) q = a.quads[a.t0 + t];
    const R* fl = reinterpret_cast<const R*>(a.fl);
    const R* fr = reinterpret_cast<const R*>(a.fr);
    // L2 look-ahead (one lane of warp 1, no shared memory): the accumulation
    // reads four function planes and updates up to four W planes after the
    // transforms, so start pulling this tile's into L2 now.  The pair-product
    // and spectrum-load passes also pull what tile (z, t + D) will load, since
    // the launch order puts that block about D waves behind this one (measured:
    // one transform ahead helps the pair-product pass; pulling ahead in the
    // accumulating pass only competes with its own read-modify-write traffic).
    if (threadIdx.x >= 32 && threadIdx.x < 64) {
        const int lane = threadIdx.x - 32;
        const int tn = t + a.lookahead;
        const bool ahead = a.lookahead > 0 && tn < (int)gridDim.y;
        if (S.tx == S.n2 && S.ty == S.n1 && lane == 0) {
            const long long off = (long long)z0 * S.n1 * S.n2;
            const uint32_t bytes = (uint32_t)((long long)S.tz * S.n1 * S.n2 * sizeof(R));
            if (bytes % 16 == 0) {
                auto planes = [&](const Quad& qq, bool with_w) {
                    prefetch_l2(fl + qq.a * N + off, bytes);
                    prefetch_l2(fr + qq.b * N + off, bytes);
                    if (qq.c >= 0) {
                        if (qq.c != qq.a) prefetch_l2(fl + qq.c * N + off, bytes);
                        prefetch_l2(fr + qq.d * N + off, bytes);
                    }
                    if (with_w) {
                        const R* wl = reinterpret_cast<const R*>(a.accl);
                        prefetch_l2(wl + qq.a * N + off, bytes);
                        if (qq.c >= 0 && qq.c != qq.a) prefetch_l2(wl + qq.c * N + off, bytes);
                        if (a.symmetric) {
                            const R* wr = reinterpret_cast<const R*>(a.accr);
                            if (qq.b != qq.a) prefetch_l2(wr + qq.b * N + off, bytes);
                            if (qq.c >= 0 && qq.d != qq.c) prefetch_l2(wr + qq.d * N + off, bytes);
                        }
                    }
                };
                if (EPI == EPI_ACCUM) planes(q, true);
                if (ahead && PRO == PRO_PAIR) planes(a.quads[a.t0 + tn], false);
            }
        }
        if (PRO == PRO_LOAD && a.bulk && ahead) {
            const Chunks ch = tile_chunks(S);
            const cx<R>* srcn = reinterpret_cast<const cx<R>*>(a.src) + (long long)tn * a.src_tstride;
            for (int k = lane; k < ch.count; k += 32) {
                long long g;
                int sk;
                chunk_at(S, k, z0, y0, x0, g, sk);
                prefetch_l2(srcn + g, (uint32_t)(ch.len * sizeof(cx<R>)));
            }
        }
    }

    // ---- prologue: global -> tile
    if (PRO == PRO_LOAD) {
        if (!bulk_in) {
            const cx<R>* src = reinterpret_cast<const cx<R>*>(a.src) + (long long)t * a.src_tstride;
            for (int e = threadIdx.x; e < tile_elems; e += S.nt()) {
                const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                tile[e] = src[((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex)];
            }
        }
    } else if (a.vec) {
        // 4 consecutive x per step; two steps in flight per thread
        const int groups = tile_elems >> 2;
        for (int g0 = threadIdx.x; g0 < groups; g0 += 2 * S.nt()) {
            V4<R> va[2], vb[2], vc[2], vd[2];
            int ee[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int g = g0 + u * S.nt();
                ee[u] = -1;
                if (g < groups) {
                    const int e = g << 2;
                    const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                    const long long r = ((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex);
                    ee[u] = e;
                    va[u] = ld4(fl + q.a * N + r);
                    if (PRO == PRO_PAIR) vb[u] = ld4(fr + q.b * N + r);
                    if (q.c >= 0) {
                        vc[u] = ld4(fl + q.c * N + r);
                        if (PRO == PRO_PAIR) vd[u] = ld4(fr + q.d * N + r);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (ee[u] < 0) continue;
                V4<R> re = PRO == PRO_PAIR ? mul4(va[u], vb[u]) : va[u];
                V4<R> im = V4<R>{R(0), R(0), R(0), R(0)};
                if (q.c >= 0) im = PRO == PRO_PAIR ? mul4(vc[u], vd[u]) : vc[u];
                tile[S.slot(ee[u])] = mk(re.x, im.x);
                tile[S.slot(ee[u] + 1)] = mk(re.y, im.y);
                tile[S.slot(ee[u] + 2)] = mk(re.z, im.z);
                tile[S.slot(ee[u] + 3)] = mk(re.w, im.w);
            }
        }
    } else {
        for (int e = threadIdx.x; e < tile_elems; e += S.nt()) {
            const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
            const long long r = ((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex);
            cx<R> v;
            if (PRO == PRO_PAIR) {
                v.re = fl[q.a * N + r] * fr[q.b * N + r];
                v.im = q.c >= 0 ? fl[q.c * N + r] * fr[q.d * N + r] : R(0);
            } else {
                v.re = fl[q.a * N + r];
                v.im = q.c >= 0 ? fl[q.c * N + r] : R(0);
            }
            tile[S.slot(e)] = v;
        }
    }
    if (bulk_in) {
        // every thread waits (bounded) for the copies; a time-out anywhere
        // makes the whole block return after the barrier
        __shared__ int timed_out;
        if (threadIdx.x == 0) timed_out = 0;
        __syncthreads();
        if (!mbar_wait_bounded(&bar, 0, a.err, 1)) timed_out = 1;
        __syncthreads();
        if (timed_out) return;
    } else {
        __syncthreads();
    }

    // ---- transforms
    if (S.axes & 1) S.template fft_x<SGN, R>(tile, twx, a);
    if (S.axes & 2) S.template fft_y<SGN, R>(tile, twy, a);
    if (S.axes & 4) {
        if (MID == MID_COULOMB) {
            S.template fft_z<-1, R>(tile, twz, a);
            const R four_pi_s = R(4.0 * 3.14159265358979323846 * a.kscale);
            const R* g1 = gt + 3 * S.n0;
            const R* g2t = gt + 3 * (S.n0 + S.n1);
            // the cut-off interaction reads its factor from the plan's table
            const R* ktab = a.kern_inline ? reinterpret_cast<const R*>(a.kern) : nullptr;
            const long long kz = (long long)S.n1 * S.n2;
            auto coulomb = [&](int e, const R* gyx, int ez, long long kyx) {
                R kv;
                if (ktab) {
                    kv = ktab[(z0 + ez) * kz + kyx];
                } else {
                    const R gx = gyx[0] + gt[3 * (z0 + ez)];
                    const R gy = gyx[1] + gt[3 * (z0 + ez) + 1];
                    const R gz = gyx[2] + gt[3 * (z0 + ez) + 2];
                    const R g2 = gx * gx + gy * gy + gz * gz;
                    kv = g2 > R(0) ? four_pi_s / g2 : R(0);
                }
                tile[e] = scale(tile[e], kv);
            };
            if (S.nt() % txy == 0) {
                // each thread keeps one (y, x) line of the tile: its G_y + G_x once
                const int l = threadIdx.x % txy, ey = l / S.tx, ex = l - ey * S.tx;
                const int xp = S.xpos(x0 + ex, y0 + ey);
                const R gyx[3] = {g1[3 * (y0 + ey)] + g2t[3 * xp], g1[3 * (y0 + ey) + 1] + g2t[3 * xp + 1],
                                  g1[3 * (y0 + ey) + 2] + g2t[3 * xp + 2]};
                const long long kyx = (long long)(y0 + ey) * S.n2 + x0 + ex;
                for (int ez = threadIdx.x / txy; ez < S.tz; ez += S.nt() / txy) coulomb(ez * txy + l, gyx, ez, kyx);
            } else {
                for (int e = threadIdx.x; e < tile_elems; e += S.nt()) {
                    const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                    const int xp = S.xpos(x0 + ex, y0 + ey);
                    const R gyx[3] = {g1[3 * (y0 + ey)] + g2t[3 * xp], g1[3 * (y0 + ey) + 1] + g2t[3 * xp + 1],
                                      g1[3 * (y0 + ey) + 2] + g2t[3 * xp + 2]};
                    coulomb(e, gyx, ez, (long long)(y0 + ey) * S.n2 + x0 + ex);
                }
            }
            __syncthreads();
            S.template fft_z<+1, R>(tile, twz, a);
        } else {
            S.template fft_z<SGN, R>(tile, twz, a);
        }
    }

    // ---- epilogue: tile -> global
    if (EPI == EPI_STORE) {
        cx<R>* dst = reinterpret_cast<cx<R>*>(a.dst) + (long long)t * a.dst_tstride;
        if (a.bulk) {
            fence_proxy_async_smem();
            __syncthreads();
            if (threadIdx.x < 32) {
                const Chunks ch = tile_chunks(S);
                for (int k = threadIdx.x; k < ch.count; k += 32) {
                    long long g;
                    int s;
                    chunk_at(S, k, z0, y0, x0, g, s);
                    bulk_store(dst + g, tile + s, (uint32_t)(ch.len * sizeof(cx<R>)));
                }
                bulk_commit();
                bulk_wait_read_all();
            }
        } else {
            for (int e = threadIdx.x; e < tile_elems; e += S.nt()) {
                const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                dst[((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex)] = tile[e];
            }
        }
        return;
    }

    R* accl = reinterpret_cast<R*>(a.accl);
    R* accr = reinterpret_cast<R*>(a.accr);
    if (EPI == EPI_SPLIT) {
        const R s = R(a.scale);
        if (a.vec) {
            for (int g = threadIdx.x; g < (tile_elems >> 2); g += S.nt()) {
                const int e = g << 2;
                const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                const long long r = ((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex);
                cx<R> v[4];
                tile_load4(S, tile, e, v);
                st4(accl + q.a * N + r, V4<R>{v[0].re * s, v[1].re * s, v[2].re * s, v[3].re * s});
                if (q.c >= 0) st4(accl + q.c * N + r, V4<R>{v[0].im * s, v[1].im * s, v[2].im * s, v[3].im * s});
            }
        } else {
            for (int e = threadIdx.x; e < tile_elems; e += S.nt()) {
                const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                const long long r = ((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex);
                accl[q.a * N + r] = tile[S.slot(e)].re * s;
                if (q.c >= 0) accl[q.c * N + r] = tile[S.slot(e)].im * s;
            }
        }
        return;
    }

    // EPI_ACCUM: W_a += v1 phi_b (+ v2 phi_d when both pairs share a), W_b += v1 f_a,
    // W_c += v2 phi_d, W_d += v2 f_c, and the pair energies sum rho v.
    R e1 = R(0), e2 = R(0);
    const bool share = q.c >= 0 && q.c == q.a;
    if (a.vec) {
        // two 4-wide float groups per round where the register budget allows
        // (<= 768 resident threads per SM: 85 registers), else one; every
        // function load of the round is issued before its first update (the
        // updates are ordered memory operations)
        constexpr int U = (sizeof(R) == 4 && Shape::kMaxThreads * Shape::kMinBlocks <= 768) ? 2 : 1;
        const int groups = tile_elems >> 2;
        for (int g0 = threadIdx.x; g0 < groups; g0 += U * S.nt()) {
            V4<R> la[U], rb[U], lc[U], rd[U];
            long long rr[U];
            int ee[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + u * S.nt();
                ee[u] = -1;
                if (g < groups) {
                    const int e = g << 2;
                    const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
                    rr[u] = ((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex);
                    ee[u] = e;
                    la[u] = ld4(fl + q.a * N + rr[u]);
                    rb[u] = ld4(fr + q.b * N + rr[u]);
                    if (q.c >= 0) {
                        lc[u] = ld4(fl + q.c * N + rr[u]);
                        rd[u] = ld4(fr + q.d * N + rr[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (ee[u] < 0) continue;
                const int e = ee[u];
                const long long r = rr[u];
                cx<R> v[4];
                tile_load4(S, tile, e, v);
                const V4<R> v1 = {v[0].re, v[1].re, v[2].re, v[3].re};
                const V4<R> v2 = {v[0].im, v[1].im, v[2].im, v[3].im};
                V4<R> wa = mul4(v1, rb[u]);
                e1 += dot4(mul4(la[u], rb[u]), v1);
                if (q.c >= 0) {
                    e2 += dot4(mul4(lc[u], rd[u]), v2);
                    if (share)
                        wa = fma4(v2, rd[u], wa);
                    else
                        red4(accl + q.c * N + r, mul4(v2, rd[u]));
                    if (a.symmetric && q.c != q.d) red4(accr + q.d * N + r, mul4(v2, lc[u]));
                }
                red4(accl + q.a * N + r, wa);
                if (a.symmetric && q.a != q.b) red4(accr + q.b * N + r, mul4(v1, la[u]));
            }
        }
    } else {
        for (int e = threadIdx.x; e < tile_elems; e += S.nt()) {
            const int ex = e % S.tx, ey = (e / S.tx) % S.ty, ez = e / txy;
            const long long r = ((long long)(z0 + ez) * S.n1 + (y0 + ey)) * S.n2 + (x0 + ex);
            const cx<R> v = tile[S.slot(e)];
            const R la = fl[q.a * N + r], rb = fr[q.b * N + r];
            e1 += la * rb * v.re;
            R wa = v.re * rb;
            if (q.c >= 0) {
                const R lc = fl[q.c * N + r], rd = fr[q.d * N + r];
                e2 += lc * rd * v.im;
                if (share)
                    wa += v.im * rd;
                else
                    atomicAdd(accl + q.c * N + r, v.im * rd);
                if (a.symmetric && q.c != q.d) atomicAdd(accr + q.d * N + r, v.im * lc);
            }
            atomicAdd(accl + q.a * N + r, wa);
            if (a.symmetric && q.a != q.b) atomicAdd(accr + q.b * N + r, v.re * la);
        }
    }
    if (a.e_part != nullptr) {
        double d1, d2;
        if constexpr (sizeof(R) == 4) {
            d1 = warp_sum_ff(e1);
            d2 = warp_sum_ff(e2);
        } else {
            d1 = double(e1);
            d2 = double(e2);
            for (int o = 16; o > 0; o >>= 1) {
                d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            }
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = S.nt() >> 5;
        if (lane == 0) {
            red[2 * warp] = d1;
            red[2 * warp + 1] = d2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s1 = 0, s2 = 0;
            for (int w = 0; w < nw; ++w) {
                s1 += red[2 * w];
                s2 += red[2 * w + 1];
            }
            double* dst = a.e_part + ((long long)(a.t0 + t) * gridDim.x + tile_id) * 2;
            dst[0] = s1;
            dst[1] = s2;
        }
    }
}


template <typename Shape, typename R, int PRO, int EPI, int MID, int SGN>
cudaError_t launch_one(const PassArgs& a, const PassShape& s, int batch, cudaStream_t st) {
    auto k = tile_pass<Shape, R, PRO, EPI, MID, SGN>;
    if (s.smem > 48 * 1024 && !stream_capturing(st)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
        if (e == cudaSuccess && Shape::kMinBlocks > 2)  // three plane blocks need the whole shared carveout
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    const int ntiles = (a.n0 / s.tz) * (a.n1 / s.ty) * (a.n2 / s.tx);
    dim3 grid(ntiles, batch);
    k<<<grid, s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

// Dispatch on (prologue, epilogue, middle, direction) for one tile geometry.
template <typename Shape, typename R>
cudaError_t dispatch(const PassArgs& a, const PassShape& s, int pro, int epi, int mid, int sgn, int batch,
                     cudaStream_t st) {
    if (mid == MID_COULOMB) return launch_one<Shape, R, PRO_LOAD, EPI_STORE, MID_COULOMB, -1>(a, s, batch, st);
    if (pro == PRO_LOAD && epi == EPI_STORE)
        return sgn < 0 ? launch_one<Shape, R, PRO_LOAD, EPI_STORE, MID_NONE, -1>(a, s, batch, st)
                       : launch_one<Shape, R, PRO_LOAD, EPI_STORE, MID_NONE, +1>(a, s, batch, st);
    if (pro == PRO_PAIR && epi == EPI_STORE && sgn < 0)
        return launch_one<Shape, R, PRO_PAIR, EPI_STORE, MID_NONE, -1>(a, s, batch, st);
    if (pro == PRO_LOAD && epi == EPI_ACCUM && sgn > 0)
        return launch_one<Shape, R, PRO_LOAD, EPI_ACCUM, MID_NONE, +1>(a, s, batch, st);
    if (pro == PRO_LOAD && epi == EPI_SPLIT && sgn > 0)
        return launch_one<Shape, R, PRO_LOAD, EPI_SPLIT, MID_NONE, +1>(a, s, batch, st);
    if (pro == PRO_PACK2 && epi == EPI_STORE && sgn < 0)
        return launch_one<Shape, R, PRO_PACK2, EPI_STORE, MID_NONE, -1>(a, s, batch, st);
    return cudaErrorInvalidValue;
}

// Cube kernels: the plane geometry carries the pair/accumulate/split/pack
// passes, the pencil geometry the load/store and Coulomb passes.  R0 != 0
// (a tuned radix plan) exists for the pair passes only: their spectrum never
// leaves them, while the orbital and W transforms keep the default plan.
template <int N, int R0 = 0>
cudaError_t dispatch_cube(const PassArgs& a, const PassShape& s, int pro, int epi, int mid, int sgn, int batch,
                          cudaStream_t st) {
    using XY = CubeShape<N, 1, N, N, cube_xy_threads(N), R0>;
    using Z = CubeShape<N, N, cube_z_ty(N), cube_z_tx(N), cube_z_threads(N), R0>;
    if (s.tz == 1 && s.ty == N && s.tx == N && s.threads == cube_xy_threads(N)) {
        if (pro == PRO_PAIR && epi == EPI_STORE && sgn < 0)
            return launch_one<XY, float, PRO_PAIR, EPI_STORE, MID_NONE, -1>(a, s, batch, st);
        if (pro == PRO_LOAD && epi == EPI_ACCUM && sgn > 0)
            return launch_one<XY, float, PRO_LOAD, EPI_ACCUM, MID_NONE, +1>(a, s, batch, st);
        if constexpr (R0 == 0) {
            if (pro == PRO_LOAD && epi == EPI_SPLIT && sgn > 0)
                return launch_one<XY, float, PRO_LOAD, EPI_SPLIT, MID_NONE, +1>(a, s, batch, st);
            if (pro == PRO_PACK2 && epi == EPI_STORE && sgn < 0)
                return launch_one<XY, float, PRO_PACK2, EPI_STORE, MID_NONE, -1>(a, s, batch, st);
        }
    } else if (s.tz == N && s.ty == cube_z_ty(N) && s.tx == cube_z_tx(N) && s.threads == cube_z_threads(N)) {
        if (mid == MID_COULOMB) return launch_one<Z, float, PRO_LOAD, EPI_STORE, MID_COULOMB, -1>(a, s, batch, st);
        if constexpr (R0 == 0) {
            if (pro == PRO_LOAD && epi == EPI_STORE)
                return sgn < 0 ? launch_one<Z, float, PRO_LOAD, EPI_STORE, MID_NONE, -1>(a, s, batch, st)
                               : launch_one<Z, float, PRO_LOAD, EPI_STORE, MID_NONE, +1>(a, s, batch, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace pass_detail
}  // namespace ace
