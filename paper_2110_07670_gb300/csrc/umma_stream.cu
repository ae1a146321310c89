// umma_stream.cu -- the two dense contractions of the ACE operator on the
// tcgen05 tensor cores, streamed from HBM (arXiv:2110.07670 Section 2.2,
// Eq. 5; the Gram is also M = Phi^T W of the construction):
//
//   Gram     G[i][j] = sum_k A[i][k] B[j][k] over K = 2 n_pw_half reals
//            (C = psi^T xi of the apply, M = Phi^T W of the build), as FP32
//            partials over K slices (about one block per SM) that
//            launch_gram_finish_f32 sums in FP64;
//   product  out[t][j] = -sum_k C[t][k] xi[k][j]  (K psi = -xi C^T), with C
//            the apply's Gram, split to TF32 hi / lo beforehand.
//
// Split precision: an FP32 operand x is carried as hi = tf32(x) and lo =
// tf32(x - hi); hi.hi goes to one TMEM accumulator and hi.lo + lo.hi to a
// second one, so every product is exact to about 2^-21 of |a||b|.  The
// tensor core's FP32 accumulation loses bits over long sums (measured: the
// error grows with the number of K = 8 steps summed in one accumulator), so
// an accumulator takes one turn of DS stages (8 K steps); then it is drained
// into FP32 sums in registers (round to nearest, one add per turn) while the
// MMAs of the next turn go to the other of two accumulator sets.
//
// Warp roles (16 warps, one block per SM; the rows of n_pw_half complex
// numbers are only 8-byte aligned, which rules out tensor-map copies for
// them):
//   warps 0-7    producers: 8-byte loads of the raw operands two 32-wide K
//                stages ahead in registers, split to TF32 hi / lo, stored in
//                the K-major 128-byte swizzle layout of one of three shared
//                buffers;
//   warps 8-15   drain a complete turn (two warps per TMEM lane quarter, 64
//                columns each) into their register sums, free the set, and
//                write the results; lane 0 of warp 8 also issues the MMAs of
//                each stage once its buffer is full, one turn ahead of its
//                own drains, and commits them (buffer free; turn complete).
// mbarriers carry every hand-off; every wait is bounded in time, sets the
// device error flag when it gives up, and makes the other roles leave.
#include <algorithm>

#include "internal.h"
#include "umma.cuh"

namespace ace {

namespace {

constexpr int TK = 32;               // K values per stage: one 128-byte swizzle row
constexpr int NB = 3;                // shared operand buffers (split, swizzled)
constexpr int DS = 2;                // stages per accumulator turn
constexpr int PF = 2;                // K stages each producer thread keeps in flight in registers (2 or 3)
constexpr int NPROD = 8;             // producer warps
constexpr int NTHR = 16 * 32;        // producers, then the drain warps
constexpr int WARP_DRAIN0 = 8;
constexpr uint32_t TMEM_COLS = 512;  // two sets of (hi.hi, small products) x 128 columns

struct __align__(1024) WsSmem {
    float a_hi[NB][128 * TK];
    float a_lo[NB][128 * TK];
    float b_hi[NB][128 * TK];
    float b_lo[NB][128 * TK];
    uint64_t full[NB];   // producers -> MMA: buffer written (NPROD arrivals)
    uint64_t empty[NB];  // MMA -> producers: buffer read (tcgen05.commit)
    uint64_t tfull[2];   // MMA -> drain: turn complete in set (tcgen05.commit)
    uint64_t tempty[2];  // drain -> MMA: set drained (8 arrivals)
    uint32_t tmem_base;
    int abort;
};

static_assert(sizeof(WsSmem) + 1024 <= 227 * 1024, "shared memory of one block (with alignment slack)");

__device__ __forceinline__ WsSmem& ws_smem() {
    extern __shared__ unsigned char smem_raw[];
    return *reinterpret_cast<WsSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
}

// full_count: arrivals that fill a buffer (the producer warps, plus one for a
// bulk copy's expected bytes)
__device__ __forceinline__ void ws_init(WsSmem& sm, int full_count) {
    if ((threadIdx.x >> 5) == 0) umma::tmem_alloc(&sm.tmem_base, TMEM_COLS);
    if (threadIdx.x == 32) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&sm.full[b], full_count);
            mbar_init(&sm.empty[b], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sm.tfull[s], 1);
            mbar_init(&sm.tempty[s], 8);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
}

// Wait for completion `use` (0, 1, ...) of a barrier, bounded in time; gives
// up at once when another role has aborted.  Returns false on either.
__device__ __forceinline__ bool ws_wait(WsSmem& sm, uint64_t* bar, long long use, int* err) {
    const uint32_t parity = (uint32_t)(use & 1);
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*reinterpret_cast<volatile int*>(&sm.abort)) return false;
        if (global_ns() - t0 > 2000000000ull) {
            if (err) atomicExch(err, 2);
            *reinterpret_cast<volatile int*>(&sm.abort) = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One producer warp finished its part of a buffer: make the generic-proxy
// stores visible to the tensor core, then one arrival for the warp.
__device__ __forceinline__ void ws_produced(uint64_t* bar) {
    fence_proxy_async_smem();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// The 12 MMAs of one stage (4 K steps x hi.hi, hi.lo, lo.hi) from buffer buf
// into accumulator set `set`.
__device__ __forceinline__ void ws_mma(WsSmem& sm, int buf, uint32_t tmem, int set, bool first) {
    constexpr uint32_t IDESC = umma::idesc_tf32(128, 128);
    const unsigned char* ah = reinterpret_cast<const unsigned char*>(sm.a_hi[buf]);
    const unsigned char* al = reinterpret_cast<const unsigned char*>(sm.a_lo[buf]);
    const unsigned char* bh = reinterpret_cast<const unsigned char*>(sm.b_hi[buf]);
    const unsigned char* bl = reinterpret_cast<const unsigned char*>(sm.b_lo[buf]);
    const uint32_t d = tmem + (uint32_t)set * 256;
#pragma unroll
    for (int kk = 0; kk < TK / 8; ++kk) {
        const uint64_t dah = umma::desc_sw128(ah + kk * 32), dal = umma::desc_sw128(al + kk * 32);
        const uint64_t dbh = umma::desc_sw128(bh + kk * 32), dbl = umma::desc_sw128(bl + kk * 32);
        const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
        umma::mma_tf32(d + 128, dal, dbh, IDESC, acc);
        umma::mma_tf32(d + 128, dah, dbl, IDESC, 1u);
        umma::mma_tf32(d, dah, dbh, IDESC, acc);
    }
}

// A drain warp's share of accumulator set `set`: its TMEM lane quarter (warp
// % 4) and its 64 columns ((warp - 8) / 4), added (or, first, stored) into
// sum[64] as hi.hi + small; then the set is released.
__device__ __forceinline__ void ws_drain(WsSmem& sm, uint32_t tmem, int set, bool first, float (&sum)[64]) {
    const int warp = threadIdx.x >> 5;
    const uint32_t taddr = tmem + (uint32_t)set * 256 + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)(((warp - WARP_DRAIN0) >> 2) * 64);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        uint32_t v[16], w[16];
        umma::tmem_ld16(taddr + 16 * h, v);
        umma::tmem_ld16(taddr + 128 + 16 * h, w);
        umma::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float x = __uint_as_float(v[c]) + __uint_as_float(w[c]);
            sum[16 * h + c] = first ? x : sum[16 * h + c] + x;
        }
    }
    umma::fence_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&sm.tempty[set]);
}

// ---------------------------------------------------------------- Gram

// Block (bx, by, bz): rows i0 .. i0 + 127 of A, rows j0 .. j0 + 127 of B,
// K range [bz kchunk, min(K, (bz + 1) kchunk)).  P[bz][i][j] = the slice's sum.
// Producer thread p owns, in every stage, the K pair 2 (p % 16) of rows
// p / 16 + 16 u (u = 0..7) of A and of B.
// ABS: the products of |A| and |B| (the s-MTACE overlap integrals).
template <bool ABS>
__global__ void __launch_bounds__(NTHR, 1)
    gram_stream(const float* __restrict__ A, const float* __restrict__ B, int m, int n, long long K, long long kchunk,
                float* __restrict__ P, int* err) {
    WsSmem& sm = ws_smem();
    const int warp = threadIdx.x >> 5;
    const int i0 = blockIdx.x * 128, j0 = blockIdx.y * 128;
    const long long k0 = (long long)blockIdx.z * kchunk;
    const long long k1 = k0 + kchunk < K ? k0 + kchunk : K;
    const int nst = (int)((k1 - k0 + TK - 1) / TK);
    const int nturn = (nst + DS - 1) / DS;
    ws_init(sm, NPROD);
    const uint32_t tmem = sm.tmem_base;

    if (warp < NPROD) {
        const int p = threadIdx.x, r0 = p >> 4, kp = 2 * (p & 15);
        unsigned valid = 0;  // bit u: row r0 + 16 u of A exists; bit 8 + u: of B
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (i0 + r0 + 16 * u < m) valid |= 1u << u;
            if (j0 + r0 + 16 * u < n) valid |= 256u << u;
        }
        const long long rs = 16 * K;  // 16 rows
        const float* pa = A + (long long)min(i0 + r0, m - 1) * K + k0 + kp;
        const float* pb = B + (long long)min(j0 + r0, n - 1) * K + k0 + kp;
        const uint32_t off = umma::sw128_offset(r0, kp);  // row r0 + 16 u: + 2048 u
        auto load = [&](float2 (&r)[16], int s) {
            const long long ko = (long long)s * TK;
            const bool in = s < nst && k0 + ko + kp < k1;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                r[u] = make_float2(0.f, 0.f);
                if (in && ((valid >> u) & 1))  // read once: cached in L2 only
                    r[u] = __ldcg(reinterpret_cast<const float2*>((u < 8 ? pa : pb) + (u & 7) * rs + ko));
            }
        };
        auto produce = [&](float2 (&r)[16], int s) -> bool {
            if (s >= nst) return true;
            const int b = s % NB;
            if (s >= NB && !ws_wait(sm, &sm.empty[b], s / NB - 1, err)) return false;
            unsigned char* ah = reinterpret_cast<unsigned char*>(sm.a_hi[b]) + off;
            unsigned char* al = reinterpret_cast<unsigned char*>(sm.a_lo[b]) + off;
            unsigned char* bh = reinterpret_cast<unsigned char*>(sm.b_hi[b]) + off;
            unsigned char* bl = reinterpret_cast<unsigned char*>(sm.b_lo[b]) + off;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                uint32_t hx, lx, hy, ly;
                umma::split_tf32(ABS ? fabsf(r[u].x) : r[u].x, hx, lx);
                umma::split_tf32(ABS ? fabsf(r[u].y) : r[u].y, hy, ly);
                *reinterpret_cast<uint2*>((u < 8 ? ah : bh) + 2048 * (u & 7)) = make_uint2(hx, hy);
                *reinterpret_cast<uint2*>((u < 8 ? al : bl) + 2048 * (u & 7)) = make_uint2(lx, ly);
            }
            load(r, s + PF);  // PF stages ahead
            ws_produced(&sm.full[b]);
            return true;
        };
        float2 ra[16], rb[16], rc[16];
        load(ra, 0);
        load(rb, 1);
        if (PF == 3) load(rc, 2);
        for (int s = 0; s < nst; s += PF)
            if (!produce(ra, s) || !produce(rb, s + 1) || (PF == 3 && !produce(rc, s + 2))) break;
    } else {
        // drain warps; lane 0 of the first also issues the MMAs, one turn
        // ahead of its own drains
        int issued = 0;
        auto issue_turn = [&](int q) -> bool {
            bool ok = true;
            if ((threadIdx.x & 31) == 0) {
                const int set = q & 1;
                if (q >= 2) ok = ws_wait(sm, &sm.tempty[set], q / 2 - 1, err);
                for (int s = q * DS; ok && s < min(nst, (q + 1) * DS); ++s) {
                    const int b = s % NB;
                    if (!(ok = ws_wait(sm, &sm.full[b], s / NB, err))) break;
                    umma::fence_after_sync();
                    ws_mma(sm, b, tmem, set, s == q * DS);
                    umma::commit(&sm.empty[b]);
                    if (s == min(nst, (q + 1) * DS) - 1) umma::commit(&sm.tfull[set]);
                    issued = s + 1;
                }
            }
            return __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
        };
        const bool issuer = warp == WARP_DRAIN0;
        float sum[64];
        bool ok = !issuer || nturn == 0 || issue_turn(0);
        for (int q = 0; q < nturn && ok; ++q) {
            if (issuer && q + 1 < nturn) ok = issue_turn(q + 1);
            if (ok) ok = ws_wait(sm, &sm.tfull[q & 1], q / 2, err);
            if (ok) {
                umma::fence_after_sync();
                ws_drain(sm, tmem, q & 1, q == 0, sum);
            }
        }
        // the MMAs in flight finish before the block releases TMEM
        if (issuer && (threadIdx.x & 31) == 0 && issued > 0)
            ws_wait(sm, &sm.empty[(issued - 1) % NB], (issued - 1) / NB, err);
        if (ok && nturn > 0) {
            const int i = i0 + (warp & 3) * 32 + (threadIdx.x & 31);
            const int jb = j0 + ((warp - WARP_DRAIN0) >> 2) * 64;
            if (i < m) {
                float* out = P + ((long long)blockIdx.z * m + i) * n;
#pragma unroll
                for (int c = 0; c < 64; ++c)
                    if (jb + c < n) out[jb + c] = sum[c];
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------- product

// out[t][j] = -sum_k C[t][k] xi[k][j].  The MMA computes the transposed tile
// D[j][t] = sum_k xi^T[j][k] C^T[k][t] (A: 128 reals of xi^T, K-major after a
// transposing store; B: 128 trials of C), so that a TMEM lane is one j and
// the stores of a warp run along j.  Tiles of 128 reals x 128 trials are
// handed out round-robin over the blocks (block b: tiles b, b + G, ...), the
// trial blocks of one j range adjacent so the second reads xi from L2; the K
// stages of 32 ACE vectors run on across tiles, and an accumulator turn never
// spans two tiles.  C comes pre-split and pre-swizzled (Cimg: per trial block
// and stage, the hi and lo shared-memory images of 16 KB each), so one bulk
// copy per half fills a stage's B operand.  Producer thread p owns, in every
// stage, xi[k0 + 4 u + (p / 8) % 4][j0 + 16 (p / 32) + 2 (p % 8) + {0, 1}]
// (u = 0..7: a warp covers 4 rows of 16 reals).
// IMG: xi comes as Ximg, its TF32 hi / lo images per 128-real tile and stage
// (xi_image_kernel), and thread 0 fills both operands of a stage with four
// bulk copies; the other producer warps have nothing to do.
template <bool IMG>
__global__ void __launch_bounds__(NTHR, 1)
    apply_product(const float* __restrict__ xi, int n, long long K, const float* __restrict__ Cimg, int nks, int T,
                  float* __restrict__ out, int* err, const float* __restrict__ Ximg) {
    WsSmem& sm = ws_smem();
    const int warp = threadIdx.x >> 5;
    const int ntb = (T + 127) / 128;
    const int ntiles = (int)((K + 127) / 128) * ntb;
    const int nsub = (nks + DS - 1) / DS;  // accumulator turns per tile
    const int G = gridDim.x;
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    const long long S = (long long)my_tiles * nks;
    ws_init(sm, IMG ? 1 : NPROD + 1);
    const uint32_t tmem = sm.tmem_base;

    if (IMG && warp < NPROD) {
        if (threadIdx.x == 0) {
            int tile = blockIdx.x, ks = 0;
            for (long long g = 0; g < S; ++g) {
                const int b = (int)(g % NB);
                if (g >= NB && !ws_wait(sm, &sm.empty[b], g / NB - 1, err)) break;
                const float* a_src = Ximg + ((long long)((tile / ntb) * nks + ks) * 2) * (128 * TK);
                const float* b_src = Cimg + ((long long)((tile % ntb) * nks + ks) * 2) * (128 * TK);
                mbar_arrive_expect_tx(&sm.full[b], 4 * 128 * TK * 4);
                bulk_load(sm.a_hi[b], a_src, 128 * TK * 4, &sm.full[b]);
                bulk_load(sm.a_lo[b], a_src + 128 * TK, 128 * TK * 4, &sm.full[b]);
                bulk_load(sm.b_hi[b], b_src, 128 * TK * 4, &sm.full[b]);
                bulk_load(sm.b_lo[b], b_src + 128 * TK, 128 * TK * 4, &sm.full[b]);
                if (++ks == nks) {
                    ks = 0;
                    tile += G;
                }
            }
        }
    } else if (warp < NPROD) {
        const int p = threadIdx.x;
        const int kq = (p >> 3) & 3, jt = (p >> 5) * 16 + (p & 7) * 2;
        const uint32_t o0 = (uint32_t)(jt * 128 + 4 * kq), o1 = o0 + 128;  // rows jt, jt + 1; + ((u ^ row % 8) << 4)
        const int x0 = jt & 7, x1 = (jt + 1) & 7;
        int tile = blockIdx.x, ks = 0;  // the stage the next load fetches
        long long lg = 0;
        auto load = [&](float2 (&r)[8]) {
#pragma unroll
            for (int u = 0; u < 8; ++u) r[u] = make_float2(0.f, 0.f);
            if (lg < S) {
                const long long j = (long long)(tile / ntb) * 128 + jt;
                const int kb = ks * TK + kq;
                const float* px = xi + (long long)kb * K + j;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (kb + 4 * u < n && j < K) r[u] = __ldg(reinterpret_cast<const float2*>(px + 4 * u * K));
                if (++ks == nks) {
                    ks = 0;
                    tile += G;
                }
            }
            ++lg;
        };
        int ctile = blockIdx.x, cks = 0;  // the stage being produced
        auto produce = [&](float2 (&r)[8], long long g) -> bool {
            if (g >= S) return true;
            const int b = (int)(g % NB);
            if (g >= NB && !ws_wait(sm, &sm.empty[b], g / NB - 1, err)) return false;
            if (p == 0) {  // C's images for this trial block and stage, by bulk copy
                const float* src = Cimg + ((long long)((ctile % ntb) * nks + cks) * 2) * (128 * TK);
                mbar_arrive_expect_tx(&sm.full[b], 2 * 128 * TK * 4);
                bulk_load(sm.b_hi[b], src, 128 * TK * 4, &sm.full[b]);
                bulk_load(sm.b_lo[b], src + 128 * TK, 128 * TK * 4, &sm.full[b]);
            }
            unsigned char* ah = reinterpret_cast<unsigned char*>(sm.a_hi[b]);
            unsigned char* al = reinterpret_cast<unsigned char*>(sm.a_lo[b]);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint32_t hx, lx, hy, ly;
                umma::split_tf32(r[u].x, hx, lx);
                umma::split_tf32(r[u].y, hy, ly);
                const uint32_t a0 = o0 + ((uint32_t)(u ^ x0) << 4), a1 = o1 + ((uint32_t)(u ^ x1) << 4);
                *reinterpret_cast<uint32_t*>(ah + a0) = hx;
                *reinterpret_cast<uint32_t*>(al + a0) = lx;
                *reinterpret_cast<uint32_t*>(ah + a1) = hy;
                *reinterpret_cast<uint32_t*>(al + a1) = ly;
            }
            load(r);  // PF stages ahead
            if (++cks == nks) {
                cks = 0;
                ctile += G;
            }
            ws_produced(&sm.full[b]);
            return true;
        };
        float2 ra[8], rb[8], rc[8];
        load(ra);
        load(rb);
        if (PF == 3) load(rc);
        for (long long g = 0; g < S; g += PF)
            if (!produce(ra, g) || !produce(rb, g + 1) || (PF == 3 && !produce(rc, g + 2))) break;
    } else {
        // drain warps; lane 0 of the first also issues the MMAs, one turn
        // ahead of its own drains.  Turn q: tile q / nsub, stages DS (q % nsub) ..
        const long long nturn = (long long)my_tiles * nsub;
        long long issued = 0;
        auto issue_turn = [&](long long q) -> bool {
            bool ok = true;
            if ((threadIdx.x & 31) == 0) {
                const int set = (int)(q & 1);
                if (q >= 2) ok = ws_wait(sm, &sm.tempty[set], q / 2 - 1, err);
                const long long g0 = (q / nsub) * nks + (q % nsub) * DS;
                const long long g1 = std::min<long long>(g0 + DS, (q / nsub + 1) * nks);
                for (long long g = g0; ok && g < g1; ++g) {
                    const int b = (int)(g % NB);
                    if (!(ok = ws_wait(sm, &sm.full[b], g / NB, err))) break;
                    umma::fence_after_sync();
                    ws_mma(sm, b, tmem, set, g == g0);
                    umma::commit(&sm.empty[b]);
                    if (g == g1 - 1) umma::commit(&sm.tfull[set]);
                    issued = g + 1;
                }
            }
            return __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
        };
        const bool issuer = warp == WARP_DRAIN0;
        float sum[64];
        const int jl = (warp & 3) * 32 + (threadIdx.x & 31);
        const int tc = ((warp - WARP_DRAIN0) >> 2) * 64;
        bool ok = !issuer || nturn == 0 || issue_turn(0);
        for (long long q = 0; q < nturn && ok; ++q) {
            if (issuer && q + 1 < nturn) ok = issue_turn(q + 1);
            if (!ok || !ws_wait(sm, &sm.tfull[q & 1], q / 2, err)) break;
            umma::fence_after_sync();
            const int sub = (int)(q % nsub);
            ws_drain(sm, tmem, (int)(q & 1), sub == 0, sum);
            if (sub == nsub - 1) {  // the tile is complete
                const int tile = blockIdx.x + (int)(q / nsub) * G;
                const long long j = (long long)(tile / ntb) * 128 + jl;
                const int t0 = (tile % ntb) * 128 + tc;
                if (j < K) {
#pragma unroll
                    for (int c = 0; c < 64; ++c)
                        if (t0 + c < T) out[(long long)(t0 + c) * K + j] = -sum[c];
                }
            }
        }
        // the MMAs in flight finish before the block releases TMEM
        if (issuer && (threadIdx.x & 31) == 0 && issued > 0)
            ws_wait(sm, &sm.empty[(issued - 1) % NB], (issued - 1) / NB, err);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TMEM_COLS);
}

// C [T][n] (double) split to TF32 hi / lo and laid out as the product's B
// operand images: Cimg[tb][ks][hi, lo][128 x 32 in the 128-byte swizzle
// layout], trials t = 128 tb + row, ACE vectors k = 32 ks + column; zero
// outside T x n.
__global__ void split_c_kernel(const double* __restrict__ C, int T, int n, int nks, float* __restrict__ Cimg) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // one (tb, ks, row, column)
    const int ntb = (T + 127) / 128;
    if (e >= (long long)ntb * nks * 128 * TK) return;
    const int col = (int)(e % TK), row = (int)((e / TK) % 128);
    const long long blk = e / (128 * TK);
    const int ks = (int)(blk % nks), tb = (int)(blk / nks);
    const int t = tb * 128 + row, k = ks * TK + col;
    float h = 0.f, l = 0.f;
    if (t < T && k < n) {
        const double c = C[(long long)t * n + k];
        h = __uint_as_float(umma::tf32_round((float)c));
        l = __uint_as_float(umma::tf32_round((float)(c - (double)h)));
    }
    float* img = Cimg + blk * 2 * (128 * TK);
    const uint32_t o = umma::sw128_offset(row, col) / 4;
    img[o] = h;
    img[128 * TK + o] = l;
}

// Ximg[jt][ks][hi, lo][128 x TK swizzled]: the TF32 split of xi^T's tile of
// reals jt * 128 .. + 127 and ACE vectors ks * TK .. + TK - 1, in the K-major
// 128-byte swizzle layout the product's A operand takes (zero past K and n).
// Thread e: one real (row, fastest, so a warp reads 32 consecutive reals of
// one vector) and 4 consecutive vectors, written as one 16-byte chunk.
__global__ void xi_image_kernel(const float* __restrict__ xi, int n, long long K, int nks, float* __restrict__ Ximg) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ntile = (K + 127) / 128;
    if (e >= ntile * nks * 128 * (TK / 4)) return;
    const int row = (int)(e % 128), kq = (int)((e / 128) % (TK / 4));
    const long long blk = e / (128 * (TK / 4));
    const int ks = (int)(blk % nks);
    const long long j = (blk / nks) * 128 + row;
    float h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = ks * TK + 4 * kq + i;
        const float x = (k < n && j < K) ? __ldg(xi + (long long)k * K + j) : 0.f;
        uint32_t hx, lx;
        umma::split_tf32(x, hx, lx);
        h[i] = __uint_as_float(hx);
        l[i] = __uint_as_float(lx);
    }
    float* img = Ximg + blk * 2 * (128 * TK);
    const uint32_t o = umma::sw128_offset(row, 4 * kq) / 4;
    *reinterpret_cast<float4*>(img + o) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(img + 128 * TK + o) = make_float4(l[0], l[1], l[2], l[3]);
}

cudaError_t set_smem(const void* k, cudaStream_t st) {
    if (stream_capturing(st)) return cudaSuccess;  // set by the same launch outside capture before
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(WsSmem) + 1024));
}

}  // namespace

long long gram_stream_kchunk(int m, int n, long long K, int sms, int max_k) {
    const long long tiles = (long long)((m + 127) / 128) * ((n + 127) / 128);
    const long long chunks = std::max<long long>(1, sms / std::max<long long>(1, tiles));
    long long kc = (K + chunks - 1) / chunks;
    if (max_k > 0) kc = std::min<long long>(kc, max_k);
    kc = (kc + TK - 1) / TK * TK;
    return std::max<long long>(kc, TK);
}

cudaError_t launch_gram_stream(const float* A, const float* B, int m, int n, long long K, long long kchunk, float* P,
                               int* err, cudaStream_t st, bool absval) {
    if (K % 2 != 0 || kchunk % TK != 0 || kchunk <= 0 || ((uintptr_t)A % 8) || ((uintptr_t)B % 8))
        return cudaErrorInvalidValue;
    cudaError_t e = set_smem(absval ? (const void*)gram_stream<true> : (const void*)gram_stream<false>, st);
    if (e != cudaSuccess) return e;
    dim3 grid((m + 127) / 128, (n + 127) / 128, (unsigned)((K + kchunk - 1) / kchunk));
    if (absval)
        gram_stream<true><<<grid, NTHR, sizeof(WsSmem) + 1024, st>>>(A, B, m, n, K, kchunk, P, err);
    else
        gram_stream<false><<<grid, NTHR, sizeof(WsSmem) + 1024, st>>>(A, B, m, n, K, kchunk, P, err);
    return cudaGetLastError();
}

size_t apply_product_scratch(int T, int n) {
    return (size_t)((T + 127) / 128) * ((n + TK - 1) / TK) * 2 * 128 * TK;
}

size_t xi_image_floats(int n, long long K) {
    return (size_t)((K + 127) / 128) * ((n + TK - 1) / TK) * 2 * 128 * TK;
}

cudaError_t launch_xi_image(const float* xi, int n, long long K, float* Ximg, cudaStream_t st) {
    if (((uintptr_t)Ximg % 16) || n < 1 || K < 1) return cudaErrorInvalidValue;
    const int nks = (n + TK - 1) / TK;
    const long long tot = (K + 127) / 128 * nks * 128 * (TK / 4);
    xi_image_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(xi, n, K, nks, Ximg);
    return cudaGetLastError();
}

cudaError_t launch_apply_product(const double* C, int T, int n, const float* xi, long long K, float* Cimg, float* out,
                                 int sms, int* err, cudaStream_t st, const float* Ximg) {
    if (K % 2 != 0 || ((uintptr_t)xi % 8) || ((uintptr_t)out % 8) || ((uintptr_t)Cimg % 16) ||
        ((uintptr_t)Ximg % 16))
        return cudaErrorInvalidValue;
    const int nks = (n + TK - 1) / TK;
    const long long tot = (long long)((T + 127) / 128) * nks * 128 * TK;
    split_c_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(C, T, n, nks, Cimg);
    const void* k = Ximg ? (const void*)apply_product<true> : (const void*)apply_product<false>;
    cudaError_t e = set_smem(k, st);
    if (e != cudaSuccess) return e;
    const long long ntiles = ((K + 127) / 128) * ((T + 127) / 128);
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(ntiles, sms));
    if (Ximg)
        apply_product<true><<<grid, NTHR, sizeof(WsSmem) + 1024, st>>>(xi, n, K, Cimg, nks, T, out, err, Ximg);
    else
        apply_product<false><<<grid, NTHR, sizeof(WsSmem) + 1024, st>>>(xi, n, K, Cimg, nks, T, out, err, nullptr);
    return cudaGetLastError();
}

}  // namespace ace
