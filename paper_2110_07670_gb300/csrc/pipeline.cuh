// pipeline.cuh -- the three pair passes of a build (Eq. 2-4) as one persistent
// kernel on the compile-time N^3 boxes with N % 16 == 0.
//
// Work items, N of each per packed transform t:
//   pass 0: plane z of t, pair product + 2-D forward FFT (transposed plane out)
//   pass 1: N z pencils of t (16 per warp), forward z, Coulomb, inverse z
//   pass 2: plane z of t, 2-D inverse FFT + exchange accumulation + energies
// Blocks stay resident and take items in ticket order from a global counter.
// Tickets are laid out in steps of 3N items; step s interleaves pass 0 of
// transform s, pass 1 of s - lag and pass 2 of s - 2 lag, so every SM mixes
// the compute-heavy transforms with the bandwidth-heavy accumulation, and a
// transform's spectrum is reused within about 2 lag steps (it stays in L2).
// Spectra live in a ring of `slots` transforms.
//
// Dependencies: pass 1 of t needs all of pass 0 of t; pass 2 of t all of pass
// 1 of t; pass 0 of t needs pass 2 of t - slots (its slot's previous user).
// Every one points to smaller tickets, held by running blocks, so the oldest
// unfinished item can always proceed.  A finished item is published by a
// block barrier, a GPU-scope fence and an atomic count; a waiting block's
// thread 0 reads the count with acquire semantics (bounded: after 2 s it sets
// the error flag and an abort flag that makes every block leave).  Spectra
// written by other blocks are read with L1-bypassing loads.
#pragma once

#include "plane.cuh"
#include "zline.cuh"

namespace ace {

namespace pipe_detail {

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float4 ld_cg4(const void* p) {
    float4 v;
    asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

// Thread 0: wait until *c >= target.  False when the kernel is aborting: the
// abort flag is set, or this wait passed 2 s (which sets the device error
// flag and the abort flag).
static __device__ __noinline__ bool wait_count(const int* c, int target, int* abort_flag, int* err) {
    if (ld_acquire(c) >= target) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        __nanosleep(128);
        if (ld_acquire(c) >= target) return true;
        if (ld_relaxed(abort_flag)) return false;
        if (global_ns() - t0 > 2000000000ull) {
            if (err) atomicExch(err, 1);
            atomicExch(abort_flag, 1);
            return false;
        }
    }
}

// Drop the lines of a dead spectrum plane from L2 without writing them back.
__device__ __forceinline__ void discard_l2(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

struct Item {
    int pass, idx, t;
};

__device__ __forceinline__ Item decode(long long tk, long long per_step, int lag) {
    Item it;
    const long long step = tk / per_step;
    const int k = (int)(tk - step * per_step);
    it.pass = k % 3;
    it.idx = k / 3;
    it.t = (int)step - it.pass * lag;
    return it;
}

// The completion count an item waits for (and its target), or null.
__device__ __forceinline__ const int* dependency(const Item& it, const PipeArgs& p) {
    if (it.t < 0 || it.t >= p.ntrans) return nullptr;
    if (it.pass == 0) return it.t >= p.slots ? p.done + 2 * p.ntrans + (it.t - p.slots) : nullptr;
    return p.done + (it.pass - 1) * p.ntrans + it.t;
}

template <int N, int F0>
__global__ void __launch_bounds__(plane_detail::Geo<N, F0>::NT, plane_detail::Geo<N, F0>::kMinBlocks)
    pair_pipeline(PassArgs a, PipeArgs p) {
    using G = plane_detail::Geo<N, F0>;
    constexpr int W = G::NT / 32;  // warps
    constexpr int GP = 16;         // pencils per warp in pass 1
    static_assert(W * GP == N, "a pass-1 item covers N pencils: N / 16 warps of 16");
    static_assert((size_t)W * N * GP <= (size_t)N * G::P, "pencil buffers fit the plane tile");
    constexpr long long NN = (long long)N * N, N3 = NN * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2 * W];
    __shared__ int s_cur;
    cx<float>* tile = reinterpret_cast<cx<float>*>(smem_raw);
    cx<float>* tw = tile + N * G::P;
    for (int j = threadIdx.x; j < N; j += G::NT) tw[j] = reinterpret_cast<const cx<float>*>(a.twx)[j];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long per_step = 3LL * N;
    const long long total = (long long)(p.ntrans + 2 * p.lag) * per_step;
    cx<float>* spec = reinterpret_cast<cx<float>*>(a.dst);
    const float* kern = reinterpret_cast<const float*>(a.kern);

    // Thread 0 runs two tickets ahead: while item i runs, ticket i + 2 is being
    // fetched and the count item i + 1 depends on is being read, so neither
    // round trip sits between items.
    long long tk_next = -1;
    if (threadIdx.x == 0) {
        long long tk = atomicAdd(p.ticket, 1);
        tk_next = p.prefetch ? atomicAdd(p.ticket, 1) : -1;
        if (tk >= total) tk = -1;
        if (tk_next >= total) tk_next = -1;
        if (tk >= 0) {
            const int* dep = dependency(decode(tk, per_step, p.lag), p);
            if (dep && !wait_count(dep, N, p.abort_flag, a.err)) tk = -1;
        }
        s_cur = (int)tk;
    }
    __syncthreads();

    for (;;) {
        const int tk = s_cur;
        if (tk < 0) break;
        const Item it = decode(tk, per_step, p.lag);
        const bool live = it.t >= 0 && it.t < p.ntrans;
        long long tk_after = -1;
        int dep_seen = 0;
        const int* dep_next = nullptr;
        if (threadIdx.x == 0 && p.prefetch) {
            tk_after = atomicAdd(p.ticket, 1);  // used at the end of this item
            if (tk_next >= 0) {
                dep_next = dependency(decode(tk_next, per_step, p.lag), p);
                if (dep_next) dep_seen = ld_relaxed(dep_next);
            }
        }
        if (live) {
            const Quad q = a.quads[a.t0 + it.t];
            cx<float>* spec_t = spec + (long long)(it.t % p.slots) * N3;
            if (it.pass == 0) {
                if (threadIdx.x == 32 && it.t + 1 < p.ntrans && (NN * 4) % 16 == 0)
                    plane_detail::prefetch_planes(a, a.quads[a.t0 + it.t + 1], it.idx * NN, (uint32_t)(NN * 4), N3,
                                                  false);
                plane_detail::pair_fwd_plane<N, false, F0>(a, q, it.idx, tile, tw, spec_t);
            } else if (it.pass == 1) {
                cx<float>* buf = tile + warp * N * GP;
                const long long p0 = (long long)(it.idx * W + warp) * GP;
                // the group's N rows of 16 values: 8 lanes x 16 bytes per row
                for (int r = lane >> 3; r < N; r += 4) {
                    const float4 v = ld_cg4(spec_t + r * NN + p0 + (lane & 7) * 2);
                    *reinterpret_cast<float4*>(buf + r * GP + (lane & 7) * 2) = v;
                }
                __syncwarp();
                zline_detail::pencils_compute<N, GP, F0>(buf, tw, kern + p0, spec_t + p0, lane);
            } else {
                const cx<float>* plane = spec_t + it.idx * NN;
                plane_detail::inv_load_cg<N, F0>(plane, tile);
                if (p.discard) {
                    __syncthreads();
                    // the plane is dead once in shared memory: drop it from L2
                    // unwritten (128-byte lines)
                    for (int l = threadIdx.x; l < (int)(NN * 8 / 128); l += G::NT)
                        discard_l2(reinterpret_cast<const char*>(plane) + (long long)l * 128);
                }
                plane_detail::inv_accum_plane<N, F0>(
                    a, q, it.idx, tile, tw, red,
                    a.e_part != nullptr ? a.e_part + ((long long)(a.t0 + it.t) * N + it.idx) * 2 : nullptr);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // publish this item (the fence also orders the early read of the
            // next item's count before its inputs are read: acquire)
            __threadfence();
            if (live) atomicAdd(p.done + it.pass * p.ntrans + it.t, 1);
            long long nxt = tk_next;
            if (!p.prefetch) {
                nxt = atomicAdd(p.ticket, 1);
                if (nxt >= total) nxt = -1;
                dep_next = nxt >= 0 ? dependency(decode(nxt, per_step, p.lag), p) : nullptr;
                dep_seen = 0;
            }
            if (nxt >= 0 && ld_relaxed(p.abort_flag)) nxt = -1;
            if (nxt >= 0 && dep_next && dep_seen < N) {
                if (!wait_count(dep_next, N, p.abort_flag, a.err)) nxt = -1;
            }
            s_cur = (int)nxt;
            tk_next = tk_after >= total ? -1 : tk_after;
        }
        __syncthreads();
    }
}

}  // namespace pipe_detail

template <int N, int F0 = 0>
cudaError_t pipeline_launch(const PassArgs& a, const PipeArgs& p, cudaStream_t st) {
    using G = plane_detail::Geo<N, F0>;
    auto k = pipe_detail::pair_pipeline<N, F0>;
    static int per_sm = [&] {
        int b = 0;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, G::NT, G::smem) != cudaSuccess)
            b = 0;
        cudaGetLastError();
        return b;
    }();
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k<<<per_sm * sms, G::NT, G::smem, st>>>(a, p);
    return cudaGetLastError();
}

}  // namespace ace
