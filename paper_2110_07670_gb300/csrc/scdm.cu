// scdm.cu -- SCDM localisation (Section 2.4) with the s'-MTACE pre-selection
// (Section 2.5): the kernels; ace_abi.cu drives them.
//
//   rho(r) = sum_i psi_i(r)^2, grad rho = 2 sum_i psi_i grad psi_i
//     (grad psi_i: transform of the coefficients i G c_i(G), exact for the
//     plane-wave expansion); every sum over orbitals in double
//   candidates: rho > <rho> and |grad rho| < <|grad rho|>, ascending grid index
//   pivots: column-pivoted QR of Psi^* on the candidate columns, as Gram-Schmidt
//     applied twice: at step k the column of largest residual norm (ties to
//     the lowest index), residual norms downdated by (q_k . a_j)^2
//   Phi = (V V^T)^{-1/2} V Psi, V[k][i] = psi_i(r_{C_k}): the polar factor of V
//     by scaled Newton-Schulz steps X <- X (3 I - X^T X) / 2 from V / |V|_F
// Sums and decisions in double; the orbitals' real-space values come in the
// plan's precision, and for single precision the QR's column pass forms its
// products in float-float arithmetic (about 2^-48 relative) on the FP32 pipes.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace ace {

namespace {

constexpr int kThreads = 256;

struct ArgMax {
    double v;
    long long j;
};

// larger value wins; equal values go to the lower index
__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
    if (b.v > a.v || (b.v == a.v && b.j >= 0 && (a.j < 0 || b.j < a.j))) return b;
    return a;
}

__device__ ArgMax block_argmax(ArgMax x) {
    __shared__ double sv[kThreads / 32];
    __shared__ long long sj[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        ArgMax y;
        y.v = __shfl_down_sync(0xffffffffu, x.v, o);
        y.j = __shfl_down_sync(0xffffffffu, x.j, o);
        x = better(x, y);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sv[w] = x.v;
        sj[w] = x.j;
    }
    __syncthreads();
    if (w == 0) {
        x.v = l < kThreads / 32 ? sv[l] : -1.0;
        x.j = l < kThreads / 32 ? sj[l] : -1;
        for (int o = 16; o > 0; o >>= 1) {
            ArgMax y;
            y.v = __shfl_down_sync(0xffffffffu, x.v, o);
            y.j = __shfl_down_sync(0xffffffffu, x.j, o);
            x = better(x, y);
        }
    }
    return x;  // valid in thread 0
}

__device__ double block_sum(double x) {
    __shared__ double s[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s[w] = x;
    __syncthreads();
    x = 0;
    if (w == 0) {
        x = l < kThreads / 32 ? s[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    }
    return x;  // valid in thread 0
}

// ------------------------------------------------------ density and gradient

template <typename R>
__global__ void deriv_coeffs_kernel(const cx<R>* __restrict__ psi, long long total, int npw,
                                    const double* __restrict__ gd, cx<R>* __restrict__ out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const R g = R(gd[e % npw]);
        const cx<R> c = psi[e];
        out[e] = mk(-g * c.im, g * c.re);  // i G_d c
    }
}

// rho[r] = sum_i phi_i(r)^2 (dphi == nullptr) or g[r] = 2 sum_i phi_i(r) dphi_i(r)
template <typename R>
__global__ void orbital_sum_kernel(const R* __restrict__ phi, const R* __restrict__ dphi, int n, long long N,
                                   double* __restrict__ out) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
        // single precision: the products of each 8 orbitals summed in float,
        // those sums in double; double precision: everything in double
        const R* b = dphi ? dphi : phi;
        double s = 0;
        for (int i0 = 0; i0 < n; i0 += 8) {
            R f = R(0);
            const int i1 = i0 + 8 < n ? i0 + 8 : n;
            for (int i = i0; i < i1; ++i) f += phi[i * N + r] * b[i * N + r];
            s += (double)f;
        }
        out[r] = dphi ? 2.0 * s : s;
    }
}

__device__ __forceinline__ double grad_norm(const double* g, long long N, long long r) {
    const double x = g[r], y = g[N + r], z = g[2 * N + r];
    return sqrt(x * x + y * y + z * z);
}

// per-block sums of rho and |grad rho| over fixed contiguous ranges
__global__ void stats_partial_kernel(const double* __restrict__ rho, const double* __restrict__ g, long long N,
                                     long long chunk, double* __restrict__ part) {
    const long long r0 = blockIdx.x * chunk, r1 = r0 + chunk < N ? r0 + chunk : N;
    double a = 0, b = 0;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        a += rho[r];
        b += grad_norm(g, N, r);
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// means[0] = <rho>, means[1] = <|grad rho|>, block partials added in order
__global__ void stats_final_kernel(const double* __restrict__ part, int nb, long long N, double* __restrict__ means) {
    if (threadIdx.x != 0) return;
    double a = 0, b = 0;
    for (int k = 0; k < nb; ++k) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    means[0] = a / (double)N;
    means[1] = b / (double)N;
}

__device__ __forceinline__ bool candidate(const double* rho, const double* g, long long N, long long r,
                                          const double* means) {
    return rho[r] > means[0] && grad_norm(g, N, r) < means[1];
}

// candidates per block of kThreads consecutive grid points
__global__ void select_count_kernel(const double* __restrict__ rho, const double* __restrict__ g, long long N,
                                    const double* __restrict__ means, int* __restrict__ counts) {
    const long long r = blockIdx.x * (long long)kThreads + threadIdx.x;
    const bool f = r < N && candidate(rho, g, N, r, means);
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// exclusive prefix sums of counts[nb] (one block), total in offsets[nb]
__global__ void select_scan_kernel(const int* __restrict__ counts, int nb, int* __restrict__ offsets) {
    __shared__ int part[kThreads];
    const int per = (nb + kThreads - 1) / kThreads;
    const int b0 = threadIdx.x * per, b1 = b0 + per < nb ? b0 + per : nb;
    int s = 0;
    for (int b = b0; b < b1; ++b) s += counts[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < kThreads; ++t) {
            const int v = part[t];
            part[t] = acc;
            acc += v;
        }
        offsets[nb] = acc;
    }
    __syncthreads();
    s = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        offsets[b] = s;
        s += counts[b];
    }
}

// the candidates' grid indices, ascending
__global__ void select_scatter_kernel(const double* __restrict__ rho, const double* __restrict__ g, long long N,
                                      const double* __restrict__ means, const int* __restrict__ offsets,
                                      int* __restrict__ sel) {
    __shared__ int wsum[kThreads / 32];
    const long long r = blockIdx.x * (long long)kThreads + threadIdx.x;
    const bool f = r < N && candidate(rho, g, N, r, means);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += wsum[k];
    if (f) sel[offsets[blockIdx.x] + before + __popc(bal & ((1u << l) - 1u))] = (int)r;
}

// A[i][s] = phi_i(r_s), r_s = sel[s] (sel == nullptr: r_s = s), in the
// orbitals' precision (the QR update reads single-precision values through
// float-float arithmetic; a float -> double conversion per product would cost
// the double-precision pipe as much as the product)
template <typename R>
__global__ void gather_columns_kernel(const R* __restrict__ phi, long long N, const int* __restrict__ sel,
                                      long long m, R* __restrict__ A) {
    const int i = blockIdx.y;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m; s += (long long)gridDim.x * blockDim.x)
        A[i * m + s] = phi[i * N + (sel ? sel[s] : s)];
}

// ------------------------------------------------------ column-pivoted QR
// Step k: (1) the pivot p_k, the column of largest residual norm nu; (2) its
// residual r = a_p - sum_{l<k} R[l][p] q_l with the coefficients R[l][j] =
// q_l . a_j stored by the earlier updates, then once more against q_0..q_{k-1}
// (classical Gram-Schmidt, twice); (3) q_k = r / |r|, R[k][j] = q_k . a_j and
// nu_j -= R[k][j]^2 for every column not chosen yet (nu < 0 marks chosen ones).

// r[i] = base - (the 8 partial sums of row i), the 8 partials held by the
// threads i % 32 of the block's 8 warps (blockDim 256)
__device__ __forceinline__ void rows_reduce8(double part, double base, double* r, int i, int n) {
    __shared__ double red[8][33];
    red[threadIdx.x >> 5][threadIdx.x & 31] = part;
    __syncthreads();
    if ((threadIdx.x >> 5) == 0 && i < n) {
        double s = 0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s += red[g][threadIdx.x];
        r[i] = base - s;
    }
}

// sum over l = g, g + 8, ... < k of c[l] Q[l][i], eight loads in flight
__device__ __forceinline__ double strided_dot8(const double* c, const double* __restrict__ Q, int n, int i, int g,
                                               int k) {
    double s[4] = {0, 0, 0, 0};
    int l = g;
    for (; l + 56 < k; l += 64) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = Q[(long long)(l + 8 * u) * n + i];
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u & 3] += c[l + 8 * u] * v[u];
    }
    for (; l < k; l += 8) s[0] += c[l] * Q[(long long)l * n + i];
    return (s[0] + s[1]) + (s[2] + s[3]);
}

// nu[j] = |a_j|^2 and the block's largest
template <typename T>
__global__ void qr_init_kernel(const T* __restrict__ A, int n, long long m, double* __restrict__ nu,
                               ArgMax* __restrict__ part) {
    ArgMax best{-1.0, -1};
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
        double s[4] = {0, 0, 0, 0};
        int i = 0;
        for (; i + 4 <= n; i += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double v = (double)A[(i + u) * m + j];
                s[u] += v * v;
            }
        for (; i < n; ++i) {
            const double v = (double)A[i * m + j];
            s[0] += v * v;
        }
        const double t = (s[0] + s[1]) + (s[2] + s[3]);
        nu[j] = t;
        best = better(best, ArgMax{t, j});
    }
    best = block_argmax(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// (1) and the first half of (2), rows [256 blockIdx.x, +256) of r.  Every
// block reduces the partials (the same result); block 0 records the pivot.
// status = 1 when the largest residual norm^2 is not above 1e-10 times the
// largest column norm^2 (nu0, recorded at step 0): the candidate columns do
// not span n_occ dimensions beyond rounding; r is then left zero.
template <typename T>
__global__ void qr_resid_kernel(const ArgMax* __restrict__ part, int nparts, const T* __restrict__ A, int n,
                                long long m, const double* __restrict__ Rrows, const double* __restrict__ Q, int k,
                                int* __restrict__ piv, double* __restrict__ nu, double* __restrict__ nu0,
                                int* __restrict__ status, double* __restrict__ r) {
    extern __shared__ double rp[];  // R[l][p], l < k
    __shared__ long long s_p;
    ArgMax best{-1.0, -1};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) best = better(best, part[b]);
    best = block_argmax(best);
    if (threadIdx.x == 0) {
        const double ref = k == 0 ? best.v : *nu0;
        const bool ok = best.j >= 0 && best.v > 1e-10 * ref && best.v == best.v;
        s_p = ok ? best.j : -1;
        if (blockIdx.x == 0) {
            if (k == 0) *nu0 = best.v;
            if (ok) {
                piv[k] = (int)best.j;
                nu[best.j] = -1.0;
            } else {
                *status = 1;
            }
        }
    }
    __syncthreads();
    const long long p = s_p;
    // 32 rows per block, the k terms of each split over 8 threads
    const int i = blockIdx.x * 32 + (threadIdx.x & 31), g = threadIdx.x >> 5;
    if (p < 0) {
        if (g == 0 && i < n) r[i] = 0.0;
        return;
    }
    for (int l = threadIdx.x; l < k; l += blockDim.x) rp[l] = Rrows[l * m + p];
    __syncthreads();
    rows_reduce8(i < n ? strided_dot8(rp, Q, n, i, g, k) : 0.0, i < n ? (double)A[i * m + p] : 0.0, r, i, n);
}

// second Gram-Schmidt pass, part 1: c_l = q_l . r, one warp per l
__global__ void qr_dots_kernel(const double* __restrict__ Q, int n, int k, const double* __restrict__ r,
                               double* __restrict__ c) {
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (l >= k) return;
    double s[4] = {0, 0, 0, 0};
    int i = lane;
    for (; i + 96 < n; i += 128)
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] += Q[(long long)l * n + i + 32 * u] * r[i + 32 * u];
    for (; i < n; i += 32) s[0] += Q[(long long)l * n + i] * r[i];
    double t = (s[0] + s[1]) + (s[2] + s[3]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) c[l] = t;
}

// part 2: r_i -= sum_l c_l q_l[i]
__global__ void qr_apply_kernel(const double* __restrict__ Q, int n, int k, const double* __restrict__ c,
                                double* __restrict__ r) {
    extern __shared__ double cs[];
    for (int l = threadIdx.x; l < k; l += blockDim.x) cs[l] = c[l];
    __syncthreads();
    const int i = blockIdx.x * 32 + (threadIdx.x & 31), g = threadIdx.x >> 5;
    rows_reduce8(i < n ? strided_dot8(cs, Q, n, i, g, k) : 0.0, i < n ? r[i] : 0.0, r, i, n);
}

// Dot product of q (double, split as qh + ql in float) with a column of
// single-precision values, in float-float arithmetic on the FP32 pipes: each
// qh a exactly as a product and its error (fmaf), ql a rounded, the running
// sum kept as an unevaluated pair (TwoSum); relative accuracy about 2^-48 of
// sum |q_i a_i|, against 2^-53 in double at a fraction of the cost on GB300.
// (The _rn intrinsics keep the rounded steps from being contracted into
// fused multiply-adds, which would break the error-free transformations.)
__device__ __forceinline__ void ff_dot_acc(float qh, float ql, float a, float& sh, float& sl) {
    const float p = __fmul_rn(qh, a);
    float e = fmaf(qh, a, -p);  // qh a - p, exactly
    e = fmaf(ql, a, e);
    const float s = __fadd_rn(sh, p), bb = __fsub_rn(s, sh);
    const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // sh + p - s, exactly
    sl = __fadd_rn(sl, __fadd_rn(t, e));
    sh = s;
}

// (3): every block normalises r itself; block 0 stores q_k and |r| = R[k][k].
// Double candidate columns: the dots in double; single-precision ones (exact
// in float): in float-float (ff_dot_acc).
template <typename T>
__global__ void qr_update_kernel(const T* __restrict__ A, int n, long long m, const double* __restrict__ r, int k,
                                 double* __restrict__ Q, double* __restrict__ Rrows, double* __restrict__ nu,
                                 double* __restrict__ rdiag, ArgMax* __restrict__ part) {
    extern __shared__ double q[];
    float* qh = reinterpret_cast<float*>(q + n);  // float-float split of q (single precision A)
    float* ql = qh + n;
    __shared__ double s_inv;
    double ss = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = r[i];
        q[i] = v;
        ss += v * v;
    }
    ss = block_sum(ss);
    if (threadIdx.x == 0) {
        s_inv = ss > 0 ? 1.0 / sqrt(ss) : 0.0;
        if (blockIdx.x == 0) rdiag[k] = sqrt(ss);  // R[k][k]
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        q[i] *= s_inv;
        if (blockIdx.x == 0) Q[(long long)k * n + i] = q[i];
        if constexpr (sizeof(T) == 4) {
            qh[i] = (float)q[i];
            ql[i] = (float)(q[i] - (double)qh[i]);
        }
    }
    __syncthreads();
    // tiles of 32 columns over one resident wave of blocks; warp g takes the
    // tile's columns (one per lane) over the row group g of 8, the groups
    // summed in shared memory
    __shared__ double red[8][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, cl = lane;
    const int rq = (n + 7) / 8, i0 = g * rq, i1 = i0 + rq < n ? i0 + rq : n;
    ArgMax best{-1.0, -1};
    double* Rk = Rrows + k * m;
    const long long ntiles = (m + 31) / 32;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long j = t * 32 + cl;
        double part_sum = 0;
        if (j < m) {
            // eight loads in flight per thread before their products
            if constexpr (sizeof(T) == 4) {
                float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f};
                int i = i0;
                for (; i + 8 <= i1; i += 8) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = (float)A[(i + u) * m + j];
#pragma unroll
                    for (int u = 0; u < 8; ++u) ff_dot_acc(qh[i + u], ql[i + u], v[u], sh[u & 1], sl[u & 1]);
                }
                for (; i < i1; ++i) ff_dot_acc(qh[i], ql[i], (float)A[i * m + j], sh[0], sl[0]);
                part_sum = ((double)sh[0] + (double)sl[0]) + ((double)sh[1] + (double)sl[1]);
            } else {
                double dd[4] = {0, 0, 0, 0};
                int i = i0;
                for (; i + 8 <= i1; i += 8) {
                    double v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = (double)A[(i + u) * m + j];
#pragma unroll
                    for (int u = 0; u < 8; ++u) dd[u & 3] += q[i + u] * v[u];
                }
                for (; i < i1; ++i) dd[0] += q[i] * (double)A[i * m + j];
                part_sum = (dd[0] + dd[1]) + (dd[2] + dd[3]);
            }
        }
        red[g][cl] = part_sum;
        __syncthreads();
        if (g == 0 && j < m) {
            double v = nu[j];
            if (v >= 0) {
                const double d = ((red[0][cl] + red[1][cl]) + (red[2][cl] + red[3][cl])) +
                                 ((red[4][cl] + red[5][cl]) + (red[6][cl] + red[7][cl]));
                Rk[j] = d;
                v -= d * d;
                if (v < 0) v = 0;
                nu[j] = v;
                best = better(best, ArgMax{v, j});
            }
        }
        __syncthreads();
    }
    best = block_argmax(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// grid point of each pivot column: out[k] = sel[piv[k]] (sel null: piv[k])
__global__ void map_pivots_kernel(const int* __restrict__ piv, const int* __restrict__ sel, int n,
                                  int* __restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = sel ? sel[piv[k]] : piv[k];
}

// ------------------------------------------------------ polar factor

// X[k][i] = A[i][piv[k]] / |V|_F, fro = |V|_F (one block)
template <typename T>
__global__ void polar_start_kernel(const T* __restrict__ A, int n, long long m, const int* __restrict__ piv,
                                   double* __restrict__ X, double* __restrict__ fro) {
    __shared__ double s_inv;
    double s = 0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int k = e / n, i = e - k * n;
        const double v = (double)A[(long long)i * m + piv[k]];
        X[e] = v;
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) {
        s_inv = 1.0 / sqrt(s);
        *fro = sqrt(s);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) X[e] *= s_inv;
}

// C = A op(B), n x n, op(B) = B^T when trans_b; 16 x 16 tiles.  err != null:
// also *err = max(*err, max |C - I|) (non-negative doubles order as their bits)
__global__ void dgemm_small_kernel(const double* __restrict__ A, const double* __restrict__ B, int n, int trans_b,
                                   double* __restrict__ C, double* __restrict__ err) {
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    double s = 0;
    for (int k0 = 0; k0 < n; k0 += 16) {
        As[ty][tx] = (row < n && k0 + tx < n) ? A[(long long)row * n + k0 + tx] : 0.0;
        const int bk = k0 + ty;
        double bv = 0;
        if (bk < n && col < n) bv = trans_b ? B[(long long)col * n + bk] : B[(long long)bk * n + col];
        Bs[ty][tx] = bv;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) s += As[ty][k] * Bs[k][tx];
        __syncthreads();
    }
    double e = 0;
    if (row < n && col < n) {
        C[(long long)row * n + col] = s;
        e = fabs(s - (row == col ? 1.0 : 0.0));
    }
    if (err) {
        for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_down_sync(0xffffffffu, e, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long*>(err), (unsigned long long)__double_as_longlong(e));
    }
}

// X <- a X + b Y
__global__ void ns_combine_kernel(double* __restrict__ X, const double* __restrict__ Y, long long total, double a,
                                  double b) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        X[e] = a * X[e] + b * Y[e];
}

int grid_for(long long items) {
    long long b = (items + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

template <typename R>
cudaError_t launch_deriv_coeffs(const cx<R>* psi, int n, int npw, const double* gd, cx<R>* out, cudaStream_t st) {
    const long long total = (long long)n * npw;
    deriv_coeffs_kernel<R><<<grid_for(total), kThreads, 0, st>>>(psi, total, npw, gd, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_orbital_sum(const R* phi, const R* dphi, int n, long long N, double* out, cudaStream_t st) {
    orbital_sum_kernel<R><<<grid_for(N), kThreads, 0, st>>>(phi, dphi, n, N, out);
    return cudaGetLastError();
}

int scdm_stats_blocks(long long N) { return (int)((N + 65535) / 65536); }

cudaError_t launch_scdm_stats(const double* rho, const double* grad, long long N, double* part, double* means,
                              cudaStream_t st) {
    const int nb = scdm_stats_blocks(N);
    stats_partial_kernel<<<nb, kThreads, 0, st>>>(rho, grad, N, 65536, part);
    stats_final_kernel<<<1, 32, 0, st>>>(part, nb, N, means);
    return cudaGetLastError();
}

int scdm_select_blocks(long long N) { return (int)((N + kThreads - 1) / kThreads); }

cudaError_t launch_scdm_select(const double* rho, const double* grad, long long N, const double* means, int* counts,
                               int* offsets, int* sel, cudaStream_t st) {
    const int nb = scdm_select_blocks(N);
    select_count_kernel<<<nb, kThreads, 0, st>>>(rho, grad, N, means, counts);
    select_scan_kernel<<<1, kThreads, 0, st>>>(counts, nb, offsets);
    select_scatter_kernel<<<nb, kThreads, 0, st>>>(rho, grad, N, means, offsets, sel);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_gather_columns(const R* phi, int n, long long N, const int* sel, long long m, R* A,
                                  cudaStream_t st) {
    dim3 grid((unsigned)std::min<long long>((m + kThreads - 1) / kThreads, 1024), (unsigned)n);
    gather_columns_kernel<R><<<grid, kThreads, 0, st>>>(phi, N, sel, m, A);
    return cudaGetLastError();
}

size_t qr_update_smem(int n) { return (size_t)n * (sizeof(double) + 2 * sizeof(float)); }

// blocks of the column passes: one per 32-column tile, at most one resident
// wave of the update kernel (its occupancy for this n times the SM count)
int scdm_qr_blocks(long long m, int n, int esz) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaError_t e =
        esz == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qr_update_kernel<float>, kThreads, qr_update_smem(n))
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qr_update_kernel<double>, kThreads, qr_update_smem(n));
    if (e != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    const long long tiles = (m + 31) / 32, wave = (long long)std::max(sms, 1) * per;
    return (int)std::max(1LL, std::min(tiles, wave));
}

size_t scdm_argmax_bytes() { return sizeof(ArgMax); }

template <typename T>
cudaError_t launch_qr_init(const T* A, int n, long long m, double* nu, void* part, cudaStream_t st) {
    qr_init_kernel<T><<<scdm_qr_blocks(m, n, sizeof(T)), kThreads, 0, st>>>(A, n, m, nu, (ArgMax*)part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qr_step(const T* A, int n, long long m, int k, QrWork w, cudaStream_t st) {
    const int rb = (n + 31) / 32, qb = scdm_qr_blocks(m, n, sizeof(T));
    qr_resid_kernel<T><<<rb, kThreads, (size_t)(k + 1) * sizeof(double), st>>>(
        (const ArgMax*)w.part, qb, A, n, m, w.R, w.Q, k, w.piv, w.nu, w.nu0, w.status, w.r);
    if (k > 0) {
        qr_dots_kernel<<<(k + 7) / 8, kThreads, 0, st>>>(w.Q, n, k, w.r, w.c);
        qr_apply_kernel<<<rb, kThreads, (size_t)k * sizeof(double), st>>>(w.Q, n, k, w.c, w.r);
    }
    qr_update_kernel<T><<<qb, kThreads, qr_update_smem(n), st>>>(
        A, n, m, w.r, k, w.Q, w.R, w.nu, w.rdiag, (ArgMax*)w.part);
    return cudaGetLastError();
}

cudaError_t launch_map_pivots(const int* piv, const int* sel, int n, int* out, cudaStream_t st) {
    map_pivots_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(piv, sel, n, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_polar_start(const T* A, int n, long long m, const int* piv, double* X, double* fro,
                               cudaStream_t st) {
    polar_start_kernel<T><<<1, kThreads, 0, st>>>(A, n, m, piv, X, fro);
    return cudaGetLastError();
}

// One scaled Newton-Schulz step X <- (alpha X) (3 I - (alpha X)^T (alpha X)) / 2,
// written as 1.5 alpha X - 0.5 alpha^3 (X X^T) X (the same map for a square
// X); err[0] = max |X X^T - I| before it.
cudaError_t launch_newton_schulz_step(double* X, double* T, double* Y, int n, double alpha, double* err,
                                      cudaStream_t st) {
    dim3 g((n + 15) / 16, (n + 15) / 16);
    cudaMemsetAsync(err, 0, sizeof(double), st);
    dgemm_small_kernel<<<g, 256, 0, st>>>(X, X, n, 1, T, err);
    dgemm_small_kernel<<<g, 256, 0, st>>>(T, X, n, 0, Y, nullptr);
    ns_combine_kernel<<<grid_for((long long)n * n), kThreads, 0, st>>>(X, Y, (long long)n * n, 1.5 * alpha,
                                                                       -0.5 * alpha * alpha * alpha);
    return cudaGetLastError();
}

template cudaError_t launch_deriv_coeffs<float>(const cx<float>*, int, int, const double*, cx<float>*, cudaStream_t);
template cudaError_t launch_deriv_coeffs<double>(const cx<double>*, int, int, const double*, cx<double>*,
                                                 cudaStream_t);
template cudaError_t launch_orbital_sum<float>(const float*, const float*, int, long long, double*, cudaStream_t);
template cudaError_t launch_orbital_sum<double>(const double*, const double*, int, long long, double*, cudaStream_t);
template cudaError_t launch_gather_columns<float>(const float*, int, long long, const int*, long long, float*,
                                                  cudaStream_t);
template cudaError_t launch_gather_columns<double>(const double*, int, long long, const int*, long long, double*,
                                                   cudaStream_t);
template cudaError_t launch_qr_init<float>(const float*, int, long long, double*, void*, cudaStream_t);
template cudaError_t launch_qr_init<double>(const double*, int, long long, double*, void*, cudaStream_t);
template cudaError_t launch_qr_step<float>(const float*, int, long long, int, QrWork, cudaStream_t);
template cudaError_t launch_qr_step<double>(const double*, int, long long, int, QrWork, cudaStream_t);
template cudaError_t launch_polar_start<float>(const float*, int, long long, const int*, double*, double*,
                                               cudaStream_t);
template cudaError_t launch_polar_start<double>(const double*, int, long long, const int*, double*, double*,
                                                cudaStream_t);

}  // namespace ace
