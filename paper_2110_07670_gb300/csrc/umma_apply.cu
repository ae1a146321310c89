// umma_apply.cu -- the two dense contractions of the ACE operator on the
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
// an accumulator takes only DS stages (8 K steps); then the block drains it
// into FP32 sums in shared memory (round to nearest, one add per drain) while
// the MMAs of the next DS stages go to the other of two accumulator sets.
//
// Data movement (the rows of n_pw_half complex numbers are only 8-byte
// aligned, which rules out tensor-map copies): 512 threads per block keep
// three 32-wide K stages of raw operands in flight in registers (8-byte
// loads, every 32-byte sector fully used), split the oldest into TF32 hi / lo
// and store it in the K-major 128-byte swizzle layout of one of two shared
// buffers while one thread issues the previous stage's MMAs; an mbarrier per
// buffer tells the threads when the tensor core has finished reading it.  One
// block per SM (about 194 KB of shared memory).  Every wait is bounded in time
// and sets the device error flag when it gives up.
#include <algorithm>

#include "internal.h"
#include "umma.cuh"

namespace ace {

namespace {

constexpr int NTHR = 512;
constexpr int TK = 32;       // K values per stage: one 128-byte swizzle row
constexpr int DS = 2;        // stages per accumulator before it is drained
constexpr int ACC_LD = 129;  // pitch of the shared FP32 sums [column][row]
constexpr uint32_t TMEM_COLS = 512;  // two sets of (hi.hi, small products) x 128 columns

struct __align__(1024) StreamSmem {
    float a_hi[2][128 * TK];
    float a_lo[2][128 * TK];
    float b_hi[2][128 * TK];
    float b_lo[2][128 * TK];
    float acc[128 * ACC_LD];  // per-thread FP32 sums of the drained accumulators
    uint64_t bar[2];
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ StreamSmem& stream_smem() {
    extern __shared__ unsigned char smem_raw[];
    return *reinterpret_cast<StreamSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void stream_init(StreamSmem& sm) {
    if ((threadIdx.x >> 5) == 0) umma::tmem_alloc(&sm.tmem_base, TMEM_COLS);
    if (threadIdx.x == 32) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        sm.abort = 0;
        fence_mbar_init();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
}

// Wait (thread 0, bounded) until the MMAs of stage g have completed, then the
// whole block; false when the wait gave up.
__device__ __forceinline__ bool stream_wait_stage(StreamSmem& sm, long long g, int* err) {
    if (threadIdx.x == 0 && !mbar_wait_bounded(&sm.bar[g & 1], (uint32_t)((g >> 1) & 1), err, 2)) sm.abort = 1;
    __syncthreads();
    umma::fence_after_sync();
    return !sm.abort;
}

// The 12 MMAs of one stage (4 K steps x hi.hi, hi.lo, lo.hi) into accumulator
// set `set`, committed to the stage's barrier (thread 0).
__device__ __forceinline__ void stream_mma(StreamSmem& sm, int buf, uint32_t tmem, int set, bool first) {
    constexpr uint32_t IDESC = umma::idesc_tf32(128, 128);
    umma::fence_after_sync();
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
    umma::commit(&sm.bar[buf]);
}

// Accumulator set `set` (hi.hi + small products): 32 columns of one TMEM lane
// per thread (warp w: lanes 32 (w % 4) .., columns 32 (w / 4) ..), 16 at a
// time, handed to f(column, value).
template <typename F>
__device__ __forceinline__ void stream_drain(uint32_t tmem, int set, F f) {
    const int warp = threadIdx.x >> 5;
    const uint32_t taddr = tmem + (uint32_t)set * 256 + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 32);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[16], w[16];
        umma::tmem_ld16(taddr + 16 * h, v);
        umma::tmem_ld16(taddr + 128 + 16 * h, w);
        umma::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) f((warp >> 2) * 32 + 16 * h + c, __uint_as_float(v[c]) + __uint_as_float(w[c]));
    }
    umma::fence_before_sync();
}

// ---------------------------------------------------------------- Gram

// Block (bx, by, bz): rows i0 .. i0 + 127 of A, rows j0 .. j0 + 127 of B,
// K range [bz kchunk, min(K, (bz + 1) kchunk)).  P[bz][i][j] = the slice's sum.
// A thread's share of a stage never changes: the K pair 2 (t % 16) of rows
// t / 16 + 32 u (u = 0..3) of A and of B, so its global pointers and shared
// offsets are formed once and advance by constant strides.
__global__ void __launch_bounds__(NTHR, 1)
    gram_stream(const float* __restrict__ A, const float* __restrict__ B, int m, int n, long long K, long long kchunk,
                float* __restrict__ P, int* err) {
    StreamSmem& sm = stream_smem();
    const int i0 = blockIdx.x * 128, j0 = blockIdx.y * 128;
    const long long k0 = (long long)blockIdx.z * kchunk;
    const long long k1 = k0 + kchunk < K ? k0 + kchunk : K;
    const int nst = (int)((k1 - k0 + TK - 1) / TK);
    const int r0 = threadIdx.x >> 4, kp = 2 * (threadIdx.x & 15);
    unsigned valid = 0;  // bit u: row r0 + 32 u of A exists; bit 4 + u: of B
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (i0 + r0 + 32 * u < m) valid |= 1u << u;
        if (j0 + r0 + 32 * u < n) valid |= 16u << u;
    }
    const long long rs = 32 * K;  // 32 rows
    const float* pa = A + (long long)min(i0 + r0, m - 1) * K + k0 + kp;
    const float* pb = B + (long long)min(j0 + r0, n - 1) * K + k0 + kp;
    const uint32_t off = umma::sw128_offset(r0, kp);  // row r0 + 32 u: + 4096 u
    float* accp = sm.acc + ((threadIdx.x >> 7) * 32) * ACC_LD + ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);
    stream_init(sm);
    const uint32_t tmem = sm.tmem_base;

    auto load = [&](float2 (&r)[8], int s) {
        const long long ko = (long long)s * TK;
        const bool in = s < nst && k0 + ko + kp < k1;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            r[u] = make_float2(0.f, 0.f);
            if (in && ((valid >> u) & 1))
                r[u] = __ldg(reinterpret_cast<const float2*>((u < 4 ? pa : pb) + (u & 3) * rs + ko));
        }
    };
    auto add_sums = [&](int set, bool first) {
        stream_drain(tmem, set, [&](int c, float v) {
            float& a = accp[(c & 31) * ACC_LD];
            a = first ? v : a + v;
        });
    };
    auto stage = [&](float2 (&r)[8], int s) -> bool {
        if (s >= nst) return true;
        const int buf = s & 1;
        // the buffer was last read by the MMAs of stage s - 2
        if (s >= 2 && !stream_wait_stage(sm, s - 2, err)) return false;
        unsigned char* ah = reinterpret_cast<unsigned char*>(sm.a_hi[buf]) + off;
        unsigned char* al = reinterpret_cast<unsigned char*>(sm.a_lo[buf]) + off;
        unsigned char* bh = reinterpret_cast<unsigned char*>(sm.b_hi[buf]) + off;
        unsigned char* bl = reinterpret_cast<unsigned char*>(sm.b_lo[buf]) + off;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            uint32_t hx, lx, hy, ly;
            umma::split_tf32(r[u].x, hx, lx);
            umma::split_tf32(r[u].y, hy, ly);
            *reinterpret_cast<uint2*>((u < 4 ? ah : bh) + 4096 * (u & 3)) = make_uint2(hx, hy);
            *reinterpret_cast<uint2*>((u < 4 ? al : bl) + 4096 * (u & 3)) = make_uint2(lx, ly);
        }
        load(r, s + 3);  // in flight during the next stages
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) stream_mma(sm, buf, tmem, (s / DS) & 1, s % DS == 0);
        // the previous DS stages are complete in the other set: drain them
        // while the tensor core works on this one
        if (s % DS == 0 && s > 0) {
            if (!stream_wait_stage(sm, s - 1, err)) return false;
            add_sums(((s - 1) / DS) & 1, s - 1 < DS);
        }
        return true;
    };

    float2 r0v[8], r1v[8], r2v[8];
    load(r0v, 0);
    load(r1v, 1);
    load(r2v, 2);
    int done = 0;  // stages whose MMAs were committed
    for (int s = 0; s < nst; s += 3) {
        if (!stage(r0v, s)) break;
        done = min(nst, s + 1);
        if (!stage(r1v, s + 1)) break;
        done = min(nst, s + 2);
        if (!stage(r2v, s + 2)) break;
        done = min(nst, s + 3);
    }
    const bool ok = !sm.abort && done == nst && done > 0;
    if (done > 0 && stream_wait_stage(sm, done - 1, err) && ok) {
        add_sums(((nst - 1) / DS) & 1, nst - 1 < DS);
        __syncthreads();
        for (int e = threadIdx.x; e < 128 * 128; e += NTHR) {
            const int i = e >> 7, j = e & 127;
            if (i0 + i < m && j0 + j < n) P[((long long)blockIdx.z * m + i0 + i) * n + j0 + j] = sm.acc[j * ACC_LD + i];
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) umma::tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------- product

// out[t][j] = -sum_k C[t][k] xi[k][j].  The MMA computes the transposed tile
// D[j][t] = sum_k xi^T[j][k] C^T[k][t] (A: 128 reals of xi^T, K-major after
// a transposing store; B: 128 trials of C), so that a TMEM lane is one j and
// the stores of a warp run along j.  Tiles of 128 reals x 128 trials are
// handed out round-robin over the blocks (block b: tiles b, b + G, ...), the
// trial blocks of one j range adjacent so the second reads xi from L2; K
// stages of 32 ACE vectors run on across tiles.  A thread's share of a stage
// is fixed: xi[k_t + 8 u][j_t, j_t + 1] (u = 0..3; a warp covers 4 rows of 16
// reals) and the 16-byte chunk t % 8 of C rows t / 8 + 64 u (u = 0, 1).
// Ch, Cl [T][np] TF32 hi / lo of C, np = n rounded up to 32 (zero padded).
__global__ void __launch_bounds__(NTHR, 1)
    apply_product(const float* __restrict__ xi, int n, long long K, const float* __restrict__ Ch,
                  const float* __restrict__ Cl, int np, int T, float* __restrict__ out, int* err) {
    StreamSmem& sm = stream_smem();
    const int ntb = (T + 127) / 128;
    const int ntiles = (int)((K + 127) / 128) * ntb;
    const int nks = np / TK;
    const int nsub = (nks + DS - 1) / DS;  // accumulator turns per tile
    const int G = gridDim.x;
    const int my_tiles = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    const long long S = (long long)my_tiles * nks;
    const int k_t = (threadIdx.x >> 8) * 4 + ((threadIdx.x >> 3) & 3);
    const int j_t = ((threadIdx.x >> 5) & 7) * 16 + (threadIdx.x & 7) * 2;
    const int t_t = threadIdx.x >> 3, c_t = threadIdx.x & 7;
    const uint32_t ox0 = umma::sw128_offset(j_t, k_t), ox1 = umma::sw128_offset(j_t + 1, k_t);  // u: ^ 32 u
    const uint32_t oc = (uint32_t)(t_t * 128 + ((c_t ^ (t_t & 7)) << 4));                        // u: + 8192 u
    const int lane_j = ((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31);  // TMEM lane of the drains
    float* accp = sm.acc + ((threadIdx.x >> 7) * 32) * ACC_LD + lane_j;
    stream_init(sm);
    const uint32_t tmem = sm.tmem_base;

    // a position in this block's stage sequence: tile (j0, t0), stage ks in it
    struct Cursor {
        long long j0;
        int t0, ks, tile;
    };
    auto set_tile = [&](Cursor& c, int tile) {
        c.tile = tile;
        c.j0 = (long long)(tile / ntb) * 128;
        c.t0 = (tile % ntb) * 128;
        c.ks = 0;
    };
    auto advance = [&](Cursor& c) {
        if (++c.ks == nks) set_tile(c, c.tile + G);
    };
    struct Regs {
        float2 x[4];
        float4 h[2], l[2];
    };
    Cursor lc;  // the stage the next load fetches
    set_tile(lc, blockIdx.x);
    long long lg = 0;
    auto load = [&](Regs& r) {
#pragma unroll
        for (int u = 0; u < 4; ++u) r.x[u] = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 2; ++u) r.h[u] = r.l[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lg < S) {
            const int kb = lc.ks * TK + k_t;
            const long long j = lc.j0 + j_t;
            const float* px = xi + (long long)kb * K + j;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (kb + 8 * u < n && j < K) r.x[u] = __ldg(reinterpret_cast<const float2*>(px + 8 * u * K));
            const long long o = (long long)(lc.t0 + t_t) * np + lc.ks * TK + c_t * 4;
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (lc.t0 + t_t + 64 * u < T) {
                    r.h[u] = __ldg(reinterpret_cast<const float4*>(Ch + o + (long long)64 * u * np));
                    r.l[u] = __ldg(reinterpret_cast<const float4*>(Cl + o + (long long)64 * u * np));
                }
            advance(lc);
        }
        ++lg;
    };
    // drain accumulator set `set` holding one turn of tile (j0, t0): into the
    // shared sums, or, at the tile's last turn, (sums +) drained values
    // negated to out
    auto drain = [&](int set, bool first, bool last, long long j0, int t0) {
        const long long j = j0 + lane_j;
        stream_drain(tmem, set, [&](int c, float v) {
            float& a = accp[(c & 31) * ACC_LD];
            const float s = first ? v : a + v;
            if (!last) {
                a = s;
            } else {
                const int t = t0 + c;
                if (j < K && t < T) out[(long long)t * K + j] = -s;
            }
        });
    };
    Cursor cc;  // the stage being issued
    set_tile(cc, blockIdx.x);
    long long pj0 = 0;  // the previous tile, drained at the first stage of the next
    int pt0 = 0;
    int turn = 0;  // accumulator turns begun
    auto stage = [&](Regs& r, long long g) -> bool {
        if (g >= S) return true;
        const int buf = (int)(g & 1);
        if (g >= 2 && !stream_wait_stage(sm, g - 2, err)) return false;
        unsigned char* ah = reinterpret_cast<unsigned char*>(sm.a_hi[buf]);
        unsigned char* al = reinterpret_cast<unsigned char*>(sm.a_lo[buf]);
        unsigned char* bh = reinterpret_cast<unsigned char*>(sm.b_hi[buf]) + oc;
        unsigned char* bl = reinterpret_cast<unsigned char*>(sm.b_lo[buf]) + oc;
        // xi[k][j], xi[k][j + 1] -> rows j, j + 1 of the K-major xi^T tile, column k
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            uint32_t hx, lx, hy, ly;
            umma::split_tf32(r.x[u].x, hx, lx);
            umma::split_tf32(r.x[u].y, hy, ly);
            *reinterpret_cast<uint32_t*>(ah + (ox0 ^ (32u * u))) = hx;
            *reinterpret_cast<uint32_t*>(al + (ox0 ^ (32u * u))) = lx;
            *reinterpret_cast<uint32_t*>(ah + (ox1 ^ (32u * u))) = hy;
            *reinterpret_cast<uint32_t*>(al + (ox1 ^ (32u * u))) = ly;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            *reinterpret_cast<float4*>(bh + 8192 * u) = r.h[u];
            *reinterpret_cast<float4*>(bl + 8192 * u) = r.l[u];
        }
        load(r);
        fence_proxy_async_smem();
        __syncthreads();
        const bool new_turn = cc.ks % DS == 0;
        if (new_turn) ++turn;
        if (threadIdx.x == 0) stream_mma(sm, buf, tmem, (turn - 1) & 1, new_turn);
        // the turn before this one is complete in the other set: drain it
        // while the tensor core works on this stage
        if (new_turn && g > 0) {
            if (!stream_wait_stage(sm, g - 1, err)) return false;
            if (cc.ks > 0)
                drain(turn & 1, cc.ks == DS, false, cc.j0, cc.t0);
            else
                drain(turn & 1, nsub == 1, true, pj0, pt0);
        }
        pj0 = cc.j0;
        pt0 = cc.t0;
        advance(cc);
        return true;
    };

    Regs q0, q1, q2;
    load(q0);
    load(q1);
    load(q2);
    long long done = 0;
    bool ok = true;
    for (long long g = 0; g < S && ok; g += 3) {
        ok = stage(q0, g);
        if (ok) done = std::min(S, g + 1);
        if (ok) ok = stage(q1, g + 1);
        if (ok) done = std::min(S, g + 2);
        if (ok) ok = stage(q2, g + 2);
        if (ok) done = std::min(S, g + 3);
    }
    const bool all = ok && !sm.abort && done == S && S > 0;
    // the last turn of the last tile
    if (done > 0 && stream_wait_stage(sm, done - 1, err) && all) drain((turn - 1) & 1, nsub == 1, true, pj0, pt0);
    umma::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) umma::tmem_dealloc(tmem, TMEM_COLS);
}

// hi / lo TF32 split of C [T][n] (double) into Ch, Cl [T][np], zero padded.
__global__ void split_c_kernel(const double* __restrict__ C, int T, int n, int np, float* __restrict__ Ch,
                               float* __restrict__ Cl) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)T * np) return;
    const int t = (int)(e / np), k = (int)(e % np);
    float h = 0.f, l = 0.f;
    if (k < n) {
        const double c = C[(long long)t * n + k];
        const uint32_t hb = umma::tf32_round((float)c);
        h = __uint_as_float(hb);
        l = __uint_as_float(umma::tf32_round((float)(c - (double)h)));
    }
    Ch[e] = h;
    Cl[e] = l;
}

cudaError_t set_smem(const void* k, cudaStream_t st) {
    if (stream_capturing(st)) return cudaSuccess;  // set by the same launch outside capture before
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(StreamSmem) + 1024));
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
                               int* err, cudaStream_t st) {
    if (K % 2 != 0 || kchunk % TK != 0 || kchunk <= 0 || ((uintptr_t)A % 8) || ((uintptr_t)B % 8))
        return cudaErrorInvalidValue;
    cudaError_t e = set_smem((const void*)gram_stream, st);
    if (e != cudaSuccess) return e;
    dim3 grid((m + 127) / 128, (n + 127) / 128, (unsigned)((K + kchunk - 1) / kchunk));
    gram_stream<<<grid, NTHR, sizeof(StreamSmem) + 1024, st>>>(A, B, m, n, K, kchunk, P, err);
    return cudaGetLastError();
}

int apply_product_np(int n) { return (n + TK - 1) / TK * TK; }

cudaError_t launch_apply_product(const double* C, int T, int n, const float* xi, long long K, float* Ch, float* Cl,
                                 float* out, int sms, int* err, cudaStream_t st) {
    if (K % 2 != 0 || ((uintptr_t)xi % 8) || ((uintptr_t)out % 8) || ((uintptr_t)Ch % 16) || ((uintptr_t)Cl % 16))
        return cudaErrorInvalidValue;
    const int np = apply_product_np(n);
    const long long tot = (long long)T * np;
    split_c_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(C, T, n, np, Ch, Cl);
    cudaError_t e = set_smem((const void*)apply_product, st);
    if (e != cudaSuccess) return e;
    const long long ntiles = ((K + 127) / 128) * ((T + 127) / 128);
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(ntiles, sms));
    apply_product<<<grid, NTHR, sizeof(StreamSmem) + 1024, st>>>(xi, n, K, Ch, Cl, np, T, out, err);
    return cudaGetLastError();
}

}  // namespace ace
