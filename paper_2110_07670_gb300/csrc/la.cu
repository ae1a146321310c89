// la.cu -- sphere scatter/gather, Gamma-point Gram products, the dense
// products of the ACE construction and apply, the FP64 Cholesky, and the
// exchange-energy reduction (arXiv:2110.07670 Section 2.2 and Eq. 4-5).
#include "internal.h"
#include "tma.cuh"

namespace ace {

namespace {

// ------------------------------------------------------------ scatter/gather

template <typename R>
__global__ void scatter_kernel(const cx<R>* __restrict__ psi, const Quad* __restrict__ quads, int t0, int npw,
                               const int* __restrict__ ip, const int* __restrict__ in, cx<R>* __restrict__ box,
                               long long N) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (p >= npw) return;
    const Quad q = quads[t0 + t];
    const cx<R> ca = psi[(long long)q.a * npw + p];
    const cx<R> cb = q.c >= 0 ? psi[(long long)q.c * npw + p] : mk(R(0), R(0));
    cx<R>* b = box + (long long)t * N;
    // Z(G) = c_a + i c_b ; Z(-G) = c_a^* + i c_b^*
    b[ip[p]] = mk(ca.re - cb.im, ca.im + cb.re);
    if (in[p] != ip[p]) b[in[p]] = mk(ca.re + cb.im, cb.re - ca.im);
}

template <typename R>
__global__ void gather_kernel(const cx<R>* __restrict__ box, const Quad* __restrict__ quads, int t0, int npw,
                              const int* __restrict__ ip, const int* __restrict__ in, long long N, R s,
                              cx<R>* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (p >= npw) return;
    const Quad q = quads[t0 + t];
    const cx<R>* b = box + (long long)t * N;
    const cx<R> z = b[ip[p]], zm = b[in[p]];
    const R h = R(0.5) * s;
    // out_a = s (Z + Zm^*)/2 ; out_c = s (Z - Zm^*)/(2i)
    out[(long long)q.a * npw + p] = mk(h * (z.re + zm.re), h * (z.im - zm.im));
    if (q.c >= 0) out[(long long)q.c * npw + p] = mk(h * (z.im + zm.im), -h * (z.re - zm.re));
}

// ---------------------------------------------------------- Gram partials
// P[c][i][j] = sum_{k in chunk c} A[i][k] B[j][k].  64 x 64 output tile per
// block, 256 threads x (4 x 4) outputs.  Products are summed in R over
// 32-wide k slices and each slice is added into double accumulators, which
// keeps float rounding to about eps * sqrt(32) of a slice.

constexpr int GT = 64, GK = 32;

template <typename R>
__global__ void __launch_bounds__(256) gram_partial_kernel(const R* __restrict__ A, const R* __restrict__ B, int m,
                                                           int n, long long K, long long kchunk, int absval,
                                                           double* __restrict__ P) {
    __shared__ R As[GK][GT + 1];
    __shared__ R Bs[GK][GT + 1];
    const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
    const long long kbeg = (long long)blockIdx.z * kchunk;
    const long long kend = kbeg + kchunk < K ? kbeg + kchunk : K;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (long long k0 = kbeg; k0 < kend; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int r = e / GK, c = e % GK;
            const long long k = k0 + c;
            R av = (i0 + r < m && k < kend) ? A[(long long)(i0 + r) * K + k] : R(0);
            R bv = (j0 + r < n && k < kend) ? B[(long long)(j0 + r) * K + k] : R(0);
            if (absval) {
                av = av < R(0) ? -av : av;
                bv = bv < R(0) ? -bv : bv;
            }
            As[c][r] = av;
            Bs[c][r] = bv;
        }
        __syncthreads();
        R s[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) s[a][b] = R(0);
#pragma unroll 8
        for (int c = 0; c < GK; ++c) {
            R av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[c][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[c][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) s[a][b] += av[a] * bv[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += double(s[a][b]);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < m && j < n) P[((long long)blockIdx.z * m + i) * n + j] = acc[a][b];
        }
}

template <typename R, typename PT>
__global__ void gram_finish_kernel(const PT* __restrict__ P, int nchunk, const R* __restrict__ A,
                                   const R* __restrict__ B, int m, int n, long long K, double* __restrict__ G,
                                   int ldg) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * n) return;
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += P[((long long)c * m + i) * n + j];
    const double g0 = double(A[(long long)i * K]) * double(B[(long long)j * K]) +
                      double(A[(long long)i * K + 1]) * double(B[(long long)j * K + 1]);
    G[(long long)i * ldg + j] = 2.0 * s - g0;
}

// The same from single-precision partials with many K slices: a block owns
// 32 consecutive elements (one per lane) and its eight warps sum interleaved
// eighths of the slices (four loads in flight each), combined in a fixed order.
__global__ void __launch_bounds__(256) gram_finish_f32_kernel(const float* __restrict__ P, int nchunk,
                                                              const float* __restrict__ A,
                                                              const float* __restrict__ B, int m, int n, long long K,
                                                              double* __restrict__ G, int ldg) {
    __shared__ double part[8][32];
    const long long tot = (long long)m * n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long e = (long long)blockIdx.x * 32 + lane;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    if (e < tot) {
        int c = w;
        for (; c + 24 < nchunk; c += 32) {
#pragma unroll
            for (int u = 0; u < 4; ++u) s[u] += (double)P[(long long)(c + 8 * u) * tot + e];
        }
        for (; c < nchunk; c += 8) s[0] += (double)P[(long long)c * tot + e];
    }
    part[w][lane] = (s[0] + s[1]) + (s[2] + s[3]);
    __syncthreads();
    if (w == 0 && e < tot) {
        double sum = 0.0;
        for (int k = 0; k < 8; ++k) sum += part[k][lane];
        const int i = (int)(e / n), j = (int)(e % n);
        const double g0 = double(A[(long long)i * K]) * double(B[(long long)j * K]) +
                          double(A[(long long)i * K + 1]) * double(B[(long long)j * K + 1]);
        G[(long long)i * ldg + j] = 2.0 * sum - g0;
    }
}

// Overlap matrix from per-chunk partials: G[i][j] = scale sum_c P[c][i][j].
template <typename PT>
__global__ void overlap_finish_kernel(const PT* __restrict__ P, int nchunk, int m, double scale,
                                      double* __restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += double(P[(long long)c * m * m + e]);
    G[e] = scale * s;
}

// ------------------------------------------------------------ NN product
// out[i][c] = alpha sum_k A[i][k] B[k][c], A double [m][k].  Block: 32 rows x
// 128 columns, 256 threads, each 4 rows x 4 columns (columns strided by 32).
// C = double: every product and sum in double (the triangular solve).
// C = float:  A rounded to float, products summed in float over 16-wide k
//             slices, slices summed in double (the ACE apply).
constexpr int NM = 32, NC = 128, NK = 16;

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    // hi + lo += x without losing the low part (Knuth's TwoSum)
    const float t = hi + x;
    const float bb = t - hi;
    lo += (hi - (t - bb)) + (x - bb);
    hi = t;
}

template <typename R, typename C>
__global__ void __launch_bounds__(256) gemm_nn_kernel(const double* __restrict__ A, int m, int kdim,
                                                      const R* __restrict__ B, long long ncols, double alpha,
                                                      R* __restrict__ out, int lower) {
    __shared__ C As[NK][NM];
    __shared__ C Bs[NK][NC];
    // row blocks vary fastest, so the blocks that share a column tile of B run together
    const int i0 = blockIdx.x * NM;
    const long long c0 = (long long)blockIdx.y * NC;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // ty: 0..7
    // double: plain double sums; float: each 16-wide slice summed in float and
    // the slices accumulated in a compensated (hi, lo) float pair
    double acc[4][4];
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[a][b] = 0.0;
            hi[a][b] = lo[a][b] = 0.f;
        }
    // a lower-triangular A has no terms beyond the block's last row
    const int kend = lower ? (kdim < i0 + NM ? kdim : i0 + NM) : kdim;
    for (int k0 = 0; k0 < kend; k0 += NK) {
        for (int e = threadIdx.x; e < NK * NM; e += 256) {
            const int r = e / NK, c = e % NK;
            As[c][r] = (i0 + r < m && k0 + c < kdim) ? C(A[(long long)(i0 + r) * kdim + k0 + c]) : C(0);
        }
        for (int e = threadIdx.x; e < NK * NC; e += 256) {
            const int r = e / NC, c = e % NC;
            Bs[r][c] = (k0 + r < kdim && c0 + c < ncols) ? C(B[(long long)(k0 + r) * ncols + c0 + c]) : C(0);
        }
        __syncthreads();
        C s[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) s[a][b] = C(0);
#pragma unroll
        for (int c = 0; c < NK; ++c) {
            C av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[c][ty + 8 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[c][tx + 32 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) s[a][b] += av[a] * bv[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if constexpr (sizeof(C) == 8)
                    acc[a][b] += double(s[a][b]);
                else
                    two_sum_acc(hi[a][b], lo[a][b], float(s[a][b]));
            }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty + 8 * a;
            const long long c = c0 + tx + 32 * b;
            const double v = sizeof(C) == 8 ? acc[a][b] : (double)hi[a][b] + (double)lo[a][b];
            if (i < m && c < ncols) out[(long long)i * ncols + c] = R(alpha * v);
        }
}

// ------------------------------------------------ Cholesky and inverse (FP64)
// -M = L L^T (right-looking, one block), then Linv = L^-1 column by column.

__global__ void __launch_bounds__(1024) neg_cholesky_inverse_kernel(const double* __restrict__ M, int n,
                                                                     double* __restrict__ L,
                                                                     double* __restrict__ Linv,
                                                                     int* __restrict__ status) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    // lower triangle of -M, symmetrised
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        L[e] = i >= j ? -0.5 * (M[(long long)i * n + j] + M[(long long)j * n + i]) : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = L[(long long)k * n + k];
            if (!(d > 0.0)) bad = 1;
            L[(long long)k * n + k] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double dkk = L[(long long)k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) L[(long long)i * n + k] /= dkk;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) L[(long long)i * n + j] -= L[(long long)i * n + k] * L[(long long)j * n + k];
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        for (int i = 0; i < j; ++i) Linv[(long long)i * n + j] = 0.0;
        Linv[(long long)j * n + j] = 1.0 / L[(long long)j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s += L[(long long)i * n + k] * Linv[(long long)k * n + j];
            Linv[(long long)i * n + j] = -s / L[(long long)i * n + i];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *status = bad;
}

// ------------------------------------------------------------ energy
__global__ void __launch_bounds__(1024) energy_reduce_kernel(const double* __restrict__ e_part,
                                                              const Quad* __restrict__ quads, int ntrans,
                                                              int ntiles, double coef, double* __restrict__ E) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int t = threadIdx.x; t < ntrans; t += blockDim.x) {
        const Quad q = quads[t];
        double e1 = 0.0, e2 = 0.0;
        for (int k = 0; k < ntiles; ++k) {
            e1 += e_part[((long long)t * ntiles + k) * 2];
            e2 += e_part[((long long)t * ntiles + k) * 2 + 1];
        }
        s += (q.a != q.b ? 2.0 : 1.0) * e1;
        if (q.c >= 0) s += (q.c != q.d ? 2.0 : 1.0) * e2;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *E = coef * red[0];
}

// The same reduction in two fixed-order stages: block b sums transforms
// b ER_T .. b ER_T + ER_T - 1 (a warp per transform, lanes over the planes)
// into out[b]; energy_final_kernel adds the block sums in order.
constexpr int ER_T = 32, ER_MAXB = 1 << 14;
__global__ void __launch_bounds__(256) energy_partial_kernel(const double* __restrict__ e_part,
                                                             const Quad* __restrict__ quads, int ntrans,
                                                             int ntiles, double* __restrict__ out) {
    __shared__ double ws[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int tt = warp; tt < ER_T; tt += 8) {
        const int t = blockIdx.x * ER_T + tt;
        if (t >= ntrans) break;
        const Quad q = quads[t];
        double e1 = 0.0, e2 = 0.0;
        for (int k = lane; k < ntiles; k += 32) {
            e1 += e_part[((long long)t * ntiles + k) * 2];
            e2 += e_part[((long long)t * ntiles + k) * 2 + 1];
        }
        for (int o = 16; o > 0; o >>= 1) {
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        }
        acc += (q.a != q.b ? 2.0 : 1.0) * e1 + (q.c >= 0 ? (q.c != q.d ? 2.0 : 1.0) * e2 : 0.0);
    }
    if (lane == 0) ws[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        out[blockIdx.x] = s;
    }
}

__global__ void energy_final_kernel(const double* __restrict__ part, int nb, double coef, double* __restrict__ E) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) s += part[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *E = coef * s;
}

// out = coef * sum_k x[k]^2 in one block, a fixed order (the fast MTS energy
// sum_t <psi_t|K psi_t> = -sum_{t,k} C_tk^2 from the apply's Gram C).
__global__ void __launch_bounds__(1024) sumsq_kernel(const double* __restrict__ x, long long n, double coef,
                                                     double* __restrict__ out) {
    __shared__ double ws[32];
    double s = 0.0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) s += x[k] * x[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        *out = coef * t;
    }
}

// -M = L L^T and L^-1 with both in shared memory (n^2 doubles, n <= 160):
// right-looking Cholesky in place, L copied out, then L^-1 in the same
// buffer, one column per thread, reading L back through L1.
__global__ void __launch_bounds__(1024) neg_cholesky_inverse_smem_kernel(const double* __restrict__ M, int n,
                                                                          double* __restrict__ L,
                                                                          double* __restrict__ Linv,
                                                                          int* __restrict__ status) {
    extern __shared__ double A[];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        A[e] = i >= j ? -0.5 * (M[(long long)i * n + j] + M[(long long)j * n + i]) : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[k * n + k];
            if (!(d > 0.0)) bad = 1;
            A[k * n + k] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double dkk = A[k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + k] /= dkk;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[i * n + j] -= A[i * n + k] * A[j * n + k];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) L[e] = A[e];
    __syncthreads();
    // column j of L^-1 by forward substitution, kept in A's column j
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
        A[j * n + j] = 1.0 / L[(long long)j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s += L[(long long)i * n + k] * A[k * n + j];
            A[i * n + j] = -s / L[(long long)i * n + i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Linv[e] = A[e];
    if (threadIdx.x == 0) *status = bad;
}

// One block waits (bounded) on an mbarrier that expects 16 bytes no copy
// will ever deliver: the time-out path of every bounded wait, without a fault
// (nothing is in flight when the block leaves).
__global__ void wait_for_nothing_kernel(int* err, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, 16);
    }
    __syncthreads();
    mbar_wait_bounded(&bar, 0, err, 1, limit_ns);
}

}  // namespace

cudaError_t launch_wait_for_nothing(int* err, int limit_ms, cudaStream_t st) {
    wait_for_nothing_kernel<<<1, 32, 0, st>>>(err, (unsigned long long)limit_ms * 1000000ull);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_scatter(const cx<R>* psi, const Quad* quads, int t0, int batch, int npw, const int* ip,
                           const int* in, cx<R>* box, long long N, cudaStream_t st) {
    dim3 grid((npw + 255) / 256, batch);
    scatter_kernel<R><<<grid, 256, 0, st>>>(psi, quads, t0, npw, ip, in, box, N);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gather(const cx<R>* box, const Quad* quads, int t0, int batch, int npw, const int* ip,
                          const int* in, long long N, double s, cx<R>* out, cudaStream_t st) {
    dim3 grid((npw + 255) / 256, batch);
    gather_kernel<R><<<grid, 256, 0, st>>>(box, quads, t0, npw, ip, in, N, R(s), out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gram_partial(const R* A, const R* B, int m, int n, long long K, int nchunk, double* P,
                                cudaStream_t st) {
    long long kc = (K + nchunk - 1) / nchunk;
    kc = (kc + GK - 1) / GK * GK;
    dim3 grid((m + GT - 1) / GT, (n + GT - 1) / GT, nchunk);
    gram_partial_kernel<R><<<grid, 256, 0, st>>>(A, B, m, n, K, kc, 0, P);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gram_finish(const double* P, int nchunk, const R* A, const R* B, int m, int n, long long K,
                               double* G, int ldg, cudaStream_t st) {
    const int tot = m * n;
    gram_finish_kernel<R, double><<<(tot + 255) / 256, 256, 0, st>>>(P, nchunk, A, B, m, n, K, G, ldg);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_overlap_partial(const R* A, int m, long long K, int nchunk, double* P, cudaStream_t st) {
    long long kc = (K + nchunk - 1) / nchunk;
    kc = (kc + GK - 1) / GK * GK;
    dim3 grid((m + GT - 1) / GT, (m + GT - 1) / GT, nchunk);
    gram_partial_kernel<R><<<grid, 256, 0, st>>>(A, A, m, m, K, kc, 1, P);
    return cudaGetLastError();
}

template <typename PT>
cudaError_t launch_overlap_finish(const PT* P, int nchunk, int m, double scale, double* G, cudaStream_t st) {
    overlap_finish_kernel<PT><<<(m * m + 255) / 256, 256, 0, st>>>(P, nchunk, m, scale, G);
    return cudaGetLastError();
}
template cudaError_t launch_overlap_finish<float>(const float*, int, int, double, double*, cudaStream_t);
template cudaError_t launch_overlap_finish<double>(const double*, int, int, double, double*, cudaStream_t);

cudaError_t launch_gram_finish_f32(const float* P, int nchunk, const float* A, const float* B, int m, int n,
                                   long long K, double* G, int ldg, cudaStream_t st) {
    const long long tot = (long long)m * n;
    gram_finish_f32_kernel<<<(unsigned)((tot + 31) / 32), 256, 0, st>>>(P, nchunk, A, B, m, n, K, G, ldg);
    return cudaGetLastError();
}

// out[i][c] = alpha sum_k A[i][k] B[k][c] with A double, B and out float, in
// float-float arithmetic on the FP32 pipes (GB300's FP64 rate is 1/64 of
// its FP32 rate): A[i][k] = ah + al as two floats, each product ah b split
// exactly into ph + pl (an FMA gives pl), al b added to the low part, and the
// running sum kept as an unevaluated float pair (hi, lo) by TwoSum.  The sum
// is good to about 2^-44 of sum |A||B| -- the double-precision form's
// accuracy once rounded to the float output.  Tiling as gemm_nn_kernel.
__global__ void __launch_bounds__(256) gemm_nn_ff_kernel(const double* __restrict__ A, int m, int kdim,
                                                         const float* __restrict__ B, long long ncols, double alpha,
                                                         float* __restrict__ out, int lower) {
    __shared__ float Ah[NK][NM], Al[NK][NM];
    __shared__ float Bs[NK][NC];
    const int i0 = blockIdx.x * NM;
    const long long c0 = (long long)blockIdx.y * NC;
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hi[a][b] = lo[a][b] = 0.f;
    const int kend = lower ? (kdim < i0 + NM ? kdim : i0 + NM) : kdim;
    for (int k0 = 0; k0 < kend; k0 += NK) {
        for (int e = threadIdx.x; e < NK * NM; e += 256) {
            const int r = e / NK, c = e % NK;
            const double v = (i0 + r < m && k0 + c < kdim) ? A[(long long)(i0 + r) * kdim + k0 + c] : 0.0;
            const float h = __double2float_rn(v);
            Ah[c][r] = h;
            Al[c][r] = __double2float_rn(v - (double)h);
        }
        for (int e = threadIdx.x; e < NK * NC; e += 256) {
            const int r = e / NC, c = e % NC;
            Bs[r][c] = (k0 + r < kdim && c0 + c < ncols) ? B[(long long)(k0 + r) * ncols + c0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < NK; ++c) {
            float ah[4], al[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                ah[a] = Ah[c][ty + 8 * a];
                al[a] = Al[c][ty + 8 * a];
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[c][tx + 32 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float ph = __fmul_rn(ah[a], bv[b]);
                    const float pl = __fmaf_rn(al[a], bv[b], __fmaf_rn(ah[a], bv[b], -ph));
                    const float t = __fadd_rn(hi[a][b], ph);
                    const float bb = __fsub_rn(t, hi[a][b]);
                    const float err = __fadd_rn(__fsub_rn(hi[a][b], __fsub_rn(t, bb)), __fsub_rn(ph, bb));
                    hi[a][b] = t;
                    lo[a][b] = __fadd_rn(lo[a][b], __fadd_rn(err, pl));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty + 8 * a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long c = c0 + tx + 32 * b;
            if (c < ncols) out[(long long)i * ncols + c] = (float)(alpha * ((double)hi[a][b] + (double)lo[a][b]));
        }
    }
}

cudaError_t launch_gemm_nn_ff(const double* A, int m, int k, const float* B, long long ncols, double alpha, float* out,
                              bool lower, cudaStream_t st) {
    dim3 grid((m + NM - 1) / NM, (unsigned)((ncols + NC - 1) / NC));
    gemm_nn_ff_kernel<<<grid, 256, 0, st>>>(A, m, k, B, ncols, alpha, out, lower ? 1 : 0);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gemm_nn(const double* A, int m, int k, const R* B, long long ncols, double alpha, R* out,
                           bool fp64_math, cudaStream_t st, bool lower) {
    dim3 grid((m + NM - 1) / NM, (unsigned)((ncols + NC - 1) / NC));
    if (fp64_math)
        gemm_nn_kernel<R, double><<<grid, 256, 0, st>>>(A, m, k, B, ncols, alpha, out, lower ? 1 : 0);
    else
        gemm_nn_kernel<R, R><<<grid, 256, 0, st>>>(A, m, k, B, ncols, alpha, out, lower ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------ blocked Cholesky
// -M = L L^T and X = L^-1 in double over many thread blocks, for the larger
// occupied sets: blocks of CB x CB, the working matrix padded to np = CB
// ceil(n / CB) with the identity outside the n x n part.  Step k of the
// right-looking factorisation: the diagonal block and its inverse T_kk in one
// block (shared memory), the panel L_ik = A_ik T_kk^T for the rows below, the
// trailing update A_ij -= L_ik L_jk^T of the lower triangle; then X by column
// blocks, X_ic = T_ii (delta_ic I - sum_{c <= j < i} L_ij X_jc).
constexpr int CB = 32;

__global__ void chol_init_kernel(const double* __restrict__ M, int n, int np, double* __restrict__ W,
                                 double* __restrict__ X, int* __restrict__ status) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0) *status = 0;
    if (e >= (long long)np * np) return;
    const int i = (int)(e / np), j = (int)(e % np);
    double v = i == j ? 1.0 : 0.0;
    if (i < n && j < n) v = i >= j ? -0.5 * (M[(long long)i * n + j] + M[(long long)j * n + i]) : 0.0;
    W[e] = v;
    X[e] = 0.0;
}

__global__ void __launch_bounds__(1024) chol_diag_kernel(double* __restrict__ W, int np, int k,
                                                         double* __restrict__ T, int* __restrict__ status) {
    __shared__ double a[CB][CB + 1], t[CB][CB + 1];
    const int r = threadIdx.x / CB, c = threadIdx.x % CB;
    double* blk = W + (long long)(k * CB) * np + k * CB;
    a[r][c] = blk[(long long)r * np + c];
    __syncthreads();
    for (int p = 0; p < CB; ++p) {
        if (threadIdx.x == 0) {
            double d = a[p][p];
            if (!(d > 0.0)) {
                atomicExch(status, 1);
                d = 1.0;
            }
            a[p][p] = sqrt(d);
        }
        __syncthreads();
        if (r > p && c == p) a[r][p] /= a[p][p];
        __syncthreads();
        if (r > p && c > p && c <= r) a[r][c] -= a[r][p] * a[c][p];
        __syncthreads();
    }
    blk[(long long)r * np + c] = c <= r ? a[r][c] : 0.0;
    if (threadIdx.x < CB) {  // column c of the inverse of the lower-triangular factor
        const int col = threadIdx.x;
        for (int i = 0; i < CB; ++i) {
            if (i < col) {
                t[i][col] = 0.0;
            } else if (i == col) {
                t[i][col] = 1.0 / a[i][i];
            } else {
                double s = 0.0;
                for (int j = col; j < i; ++j) s += a[i][j] * t[j][col];
                t[i][col] = -s / a[i][i];
            }
        }
    }
    __syncthreads();
    T[(long long)k * CB * CB + r * CB + c] = t[r][c];
}

__global__ void __launch_bounds__(1024) chol_panel_kernel(double* __restrict__ W, int np, int k,
                                                          const double* __restrict__ T) {
    __shared__ double a[CB][CB + 1], t[CB][CB + 1];
    const int r = threadIdx.x / CB, c = threadIdx.x % CB;
    const int i = k + 1 + blockIdx.x;
    double* blk = W + (long long)(i * CB) * np + k * CB;
    a[r][c] = blk[(long long)r * np + c];
    t[r][c] = T[(long long)k * CB * CB + r * CB + c];
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q <= c; ++q) s += a[r][q] * t[c][q];  // (A T^T)[r][c], T lower triangular
    __syncthreads();
    blk[(long long)r * np + c] = s;
}

__global__ void __launch_bounds__(1024) chol_update_kernel(double* __restrict__ W, int np, int k) {
    __shared__ double li[CB][CB + 1], lj[CB][CB + 1];
    const int r = threadIdx.x / CB, c = threadIdx.x % CB;
    // lower-triangle tile (ii, jj), jj <= ii, of the trailing matrix
    const int tb = blockIdx.x;
    int ii = (int)((sqrt(8.0 * tb + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= tb) ++ii;
    while (ii * (ii + 1) / 2 > tb) --ii;
    const int jj = tb - ii * (ii + 1) / 2;
    const int i = k + 1 + ii, j = k + 1 + jj;
    li[r][c] = W[(long long)(i * CB + r) * np + k * CB + c];
    lj[r][c] = W[(long long)(j * CB + r) * np + k * CB + c];
    __syncthreads();
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < CB; ++q) s += li[r][q] * lj[c][q];
    W[(long long)(i * CB + r) * np + j * CB + c] -= s;
}

__global__ void __launch_bounds__(1024) chol_inverse_kernel(const double* __restrict__ W, int np,
                                                            const double* __restrict__ T, double* __restrict__ X) {
    __shared__ double l[CB][CB + 1], x[CB][CB + 1], s[CB][CB + 1];
    const int r = threadIdx.x / CB, cc = threadIdx.x % CB;
    const int nb = np / CB, c = blockIdx.x;
    for (int i = c; i < nb; ++i) {
        double acc = (i == c && r == cc) ? 1.0 : 0.0;
        for (int j = c; j < i; ++j) {
            l[r][cc] = W[(long long)(i * CB + r) * np + j * CB + cc];
            x[r][cc] = X[(long long)(j * CB + r) * np + c * CB + cc];  // written by this block at row block j
            __syncthreads();
#pragma unroll 8
            for (int q = 0; q < CB; ++q) acc -= l[r][q] * x[q][cc];
            __syncthreads();
        }
        s[r][cc] = acc;
        l[r][cc] = T[(long long)i * CB * CB + r * CB + cc];
        __syncthreads();
        double v = 0.0;
        for (int q = 0; q <= r; ++q) v += l[r][q] * s[q][cc];
        X[(long long)(i * CB + r) * np + c * CB + cc] = v;
        __syncthreads();
    }
}

__global__ void chol_extract_kernel(const double* __restrict__ W, const double* __restrict__ X, int n, int np,
                                    double* __restrict__ L, double* __restrict__ Linv) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    L[e] = j <= i ? W[(long long)i * np + j] : 0.0;
    Linv[e] = j <= i ? X[(long long)i * np + j] : 0.0;
}

size_t neg_cholesky_work(int n) {
    const size_t np = (size_t)(n + CB - 1) / CB * CB;
    return 2 * np * np + np * CB;
}

cudaError_t launch_neg_cholesky_blocked(const double* M, int n, double* L, double* Linv, int* status, double* work,
                                        int* nlaunch, cudaStream_t st) {
    const int np = (n + CB - 1) / CB * CB, nb = np / CB;
    double* W = work;
    double* X = work + (size_t)np * np;
    double* T = X + (size_t)np * np;
    int count = 0;
    chol_init_kernel<<<(unsigned)(((long long)np * np + 255) / 256), 256, 0, st>>>(M, n, np, W, X, status);
    ++count;
    for (int k = 0; k < nb; ++k) {
        chol_diag_kernel<<<1, CB * CB, 0, st>>>(W, np, k, T, status);
        ++count;
        const int m = nb - k - 1;
        if (m > 0) {
            chol_panel_kernel<<<m, CB * CB, 0, st>>>(W, np, k, T);
            chol_update_kernel<<<m * (m + 1) / 2, CB * CB, 0, st>>>(W, np, k);
            count += 2;
        }
    }
    chol_inverse_kernel<<<nb, CB * CB, 0, st>>>(W, np, T, X);
    chol_extract_kernel<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, st>>>(W, X, n, np, L, Linv);
    count += 2;
    if (nlaunch) *nlaunch = count;
    return cudaGetLastError();
}

cudaError_t launch_neg_cholesky_inverse(const double* M, int n, double* L, double* Linv, int* status,
                                        cudaStream_t st) {
    const size_t smem = (size_t)n * n * sizeof(double);
    if (smem <= 200 * 1024) {
        static const cudaError_t attr = cudaFuncSetAttribute(
            neg_cholesky_inverse_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (attr != cudaSuccess) return attr;
        neg_cholesky_inverse_smem_kernel<<<1, 1024, smem, st>>>(M, n, L, Linv, status);
    } else {
        neg_cholesky_inverse_kernel<<<1, 1024, 0, st>>>(M, n, L, Linv, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const double* x, long long n, double coef, double* out, cudaStream_t st) {
    sumsq_kernel<<<1, 1024, 0, st>>>(x, n, coef, out);
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const double* e_part, const Quad* quads, int ntrans, int ntiles, double coef,
                                 double* E, cudaStream_t st) {
    // stage 1: blocks of ER_T transforms into per-block sums (in E[1 ..]);
    // stage 2: one warp adds them in block order
    const int nb = std::max(1, (ntrans + ER_T - 1) / ER_T);
    if (nb > ER_MAXB) {
        energy_reduce_kernel<<<1, 1024, 0, st>>>(e_part, quads, ntrans, ntiles, coef, E);
        return cudaGetLastError();
    }
    energy_partial_kernel<<<nb, 256, 0, st>>>(e_part, quads, ntrans, ntiles, E + 1);
    energy_final_kernel<<<1, 32, 0, st>>>(E + 1, nb, coef, E);
    return cudaGetLastError();
}

#define ACE_INST(R)                                                                                             \
    template cudaError_t launch_scatter<R>(const cx<R>*, const Quad*, int, int, int, const int*, const int*,   \
                                           cx<R>*, long long, cudaStream_t);                                    \
    template cudaError_t launch_gather<R>(const cx<R>*, const Quad*, int, int, int, const int*, const int*,    \
                                          long long, double, cx<R>*, cudaStream_t);                             \
    template cudaError_t launch_gram_partial<R>(const R*, const R*, int, int, long long, int, double*,          \
                                                cudaStream_t);                                                  \
    template cudaError_t launch_gram_finish<R>(const double*, int, const R*, const R*, int, int, long long,     \
                                               double*, int, cudaStream_t);                                     \
    template cudaError_t launch_gemm_nn<R>(const double*, int, int, const R*, long long, double, R*, bool,      \
                                           cudaStream_t, bool);                                                 \
    template cudaError_t launch_overlap_partial<R>(const R*, int, long long, int, double*, cudaStream_t);
ACE_INST(float)
ACE_INST(double)
#undef ACE_INST

}  // namespace ace
