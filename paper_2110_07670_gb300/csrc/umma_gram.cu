// umma_gram.cu -- the s-MTACE overlap S_ij = (Omega / N) sum_r |phi_i(r)| |phi_j(r)|
// (arXiv:2110.07670 Section 2.4) as a Gram product of |phi| on the tcgen05
// tensor cores.
//
// Split precision: every FP32 operand x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi), and the four products hi.hi + hi.lo + lo.hi + lo.lo
// are accumulated in FP32 in tensor memory (TMEM) by tcgen05.mma kind::tf32,
// which carries the product to about 2^-22 of |a||b|.  Each thread block owns
// a 128 x 128 output tile and one K slice of grid points; the large products
// (hi.hi) and the three small ones accumulate in separate TMEM accumulators,
// the slice's partial is written in single precision and the slices are
// summed in double by launch_overlap_finish (la.cu).
//
// Data movement: the block's threads load 128 x 32 FP32 slices of the
// real-space orbitals as 8-byte vectors, split them and store hi / lo in the
// K-major 128-byte swizzle layout (the next slice is already loading into
// registers while the tensor core works); one thread issues the MMAs and
// commits them to an mbarrier; tcgen05.ld drains the accumulators.  64 KB of
// shared memory and 256 TMEM columns let two blocks share an SM.  Every wait
// is bounded in time and sets the plan's device error flag when it gives up.
#include <cstdio>

#include "internal.h"
#include "umma.cuh"

namespace ace {

namespace {

constexpr int TM = 128, TN = 128, TK = 32;   // output tile, K per stage (one 128-byte swizzle row)
constexpr int KCHUNK = 128;                   // K per block
constexpr uint32_t TMEM_COLS = 256;  // two 128-column FP32 accumulators

struct __align__(1024) GramSmem {
    float a_hi[TM * TK];
    float a_lo[TM * TK];
    float b_hi[TN * TK];
    float b_lo[TN * TK];
    uint64_t mma_done;
    uint32_t tmem_base;
    int abort;
};

// instruction descriptor: D f32, A/B tf32, both K-major, M = TM, N = TN
constexpr uint32_t kIdesc = umma::idesc_tf32(TM, TN);
using umma::sw128_offset;
using umma::tf32_round;
using umma::tmem_ld32;

__device__ __forceinline__ uint64_t smem_desc_sw128(const void* p) { return umma::desc_sw128(p); }

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    umma::mma_tf32(d_tmem, a, b, kIdesc, accumulate);
}

constexpr int NTHR = 256;

__global__ void __launch_bounds__(NTHR, 2)
    gram_partial_umma(const float* __restrict__ A, const float* __restrict__ B, int m, int n, long long K,
                      long long kchunk, int absval, float* __restrict__ P, int* err) {
    extern __shared__ unsigned char smem_raw[];
    GramSmem& sm = *reinterpret_cast<GramSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
    const long long k0 = (long long)blockIdx.z * kchunk;
    const int nst = (int)(((K - k0 < kchunk ? K - k0 : kchunk) + TK - 1) / TK);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        mbar_init(&sm.mma_done, 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem_base;

    // Each thread owns 16 float2 of a stage (8 of A, 8 of B); the next stage is
    // loaded into registers while the tensor core works on the current one.
    constexpr int PER = 2 * TM * (TK / 2) / NTHR;  // 16
    float2 x[PER];
    auto load_stage = [&](int s) {
        const long long kb = k0 + (long long)s * TK;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * NTHR;
            const bool isb = e >= TM * (TK / 2);
            const int ee = isb ? e - TM * (TK / 2) : e;
            const int row = ee / (TK / 2), k = 2 * (ee % (TK / 2));
            const int grow = (isb ? j0 : i0) + row;
            const long long gk = kb + k;
            x[u] = make_float2(0.f, 0.f);
            if (grow < (isb ? n : m) && gk < K) {
                const float* src = (isb ? B : A) + (long long)grow * K + gk;
                if (gk + 1 < K)
                    x[u] = __ldg(reinterpret_cast<const float2*>(src));
                else
                    x[u].x = __ldg(src);
                if (absval) {
                    x[u].x = fabsf(x[u].x);
                    x[u].y = fabsf(x[u].y);
                }
            }
        }
    };
    unsigned char* ah = reinterpret_cast<unsigned char*>(sm.a_hi);
    unsigned char* al = reinterpret_cast<unsigned char*>(sm.a_lo);
    unsigned char* bh = reinterpret_cast<unsigned char*>(sm.b_hi);
    unsigned char* bl = reinterpret_cast<unsigned char*>(sm.b_lo);
    load_stage(0);
    int committed = 0;
    for (int s = 0; s < nst; ++s) {
        // the single operand buffer was last read by the MMAs of stage s - 1
        if (s >= 1 && !mbar_wait_bounded(&sm.mma_done, (s - 1) & 1, err, 2)) sm.abort = 1;
        __syncthreads();
        if (sm.abort) break;
        // split hi = tf32(x), lo = tf32(x - hi) and store in the swizzled layout
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * NTHR;
            const bool isb = e >= TM * (TK / 2);
            const int ee = isb ? e - TM * (TK / 2) : e;
            const int row = ee / (TK / 2), k = 2 * (ee % (TK / 2));
            const uint32_t hx = tf32_round(x[u].x), hy = tf32_round(x[u].y);
            const uint32_t lx = tf32_round(x[u].x - __uint_as_float(hx)), ly = tf32_round(x[u].y - __uint_as_float(hy));
            const uint32_t off = sw128_offset(row, k);
            *reinterpret_cast<uint2*>((isb ? bh : ah) + off) = make_uint2(hx, hy);
            *reinterpret_cast<uint2*>((isb ? bl : al) + off) = make_uint2(lx, ly);
        }
        if (s + 1 < nst) load_stage(s + 1);  // in flight during this stage's MMAs
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TK / 8; ++kk) {
                // advance 8 tf32 (32 bytes) along K inside the swizzle row
                const uint64_t dah = smem_desc_sw128(ah + kk * 32), dal = smem_desc_sw128(al + kk * 32);
                const uint64_t dbh = smem_desc_sw128(bh + kk * 32), dbl = smem_desc_sw128(bl + kk * 32);
                const uint32_t acc0 = (s > 0 || kk > 0) ? 1u : 0u;
                // the three small products in their own accumulator, so the
                // large one is rounded once per K step only
                umma_tf32(tmem + TN, dal, dbl, acc0);
                umma_tf32(tmem + TN, dal, dbh, 1u);
                umma_tf32(tmem + TN, dah, dbl, 1u);
                umma_tf32(tmem, dah, dbh, acc0);
            }
            umma::commit(&sm.mma_done);
        }
        ++committed;
    }
    __syncthreads();
    const bool ok = !sm.abort;
    if (committed > 0) {
        if (!mbar_wait_bounded(&sm.mma_done, (committed - 1) & 1, err, 2)) sm.abort = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (ok && !sm.abort && committed == nst) {
        // warp w reads TMEM lanes 32 (w % 4) .. +31 (output rows), columns
        // 64 (w / 4) .. +63, 32 at a time
        const int row = i0 + (warp & 3) * 32 + lane;
        float* out = P + ((long long)blockIdx.z * m + row) * n;
        for (int c0 = (warp >> 2) * 64; c0 < (warp >> 2) * 64 + 64; c0 += 32) {
            uint32_t v[32], w[32];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
            tmem_ld32(taddr + TN, w);
            tmem_ld32(taddr, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < m) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (j0 + c0 + c < n) out[j0 + c0 + c] = __uint_as_float(v[c]) + __uint_as_float(w[c]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

cudaError_t launch_overlap_partial_umma(const float* A, int m, long long K, long long kchunk, float* P, int* err,
                                        cudaStream_t st) {
    if (K % 2 != 0 || kchunk % TK != 0 || kchunk <= 0 || ((uintptr_t)A % 8)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(GramSmem) + 1024;
    cudaError_t e = cudaFuncSetAttribute(gram_partial_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((m + TM - 1) / TM, (m + TM - 1) / TM, (unsigned)((K + kchunk - 1) / kchunk));
    gram_partial_umma<<<grid, NTHR, smem, st>>>(A, A, m, m, K, kchunk, 1, P, err);
    return cudaGetLastError();
}

}  // namespace ace
