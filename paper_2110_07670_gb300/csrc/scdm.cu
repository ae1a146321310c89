// scdm.cu -- SCDM localisation (Section 2.4) with the s'-MTACE pre-selection
// (Section 2.5): the kernels; ace_abi.cu drives them.
//
//   rho(r) = sum_i psi_i(r)^2, grad rho = 2 sum_i psi_i grad psi_i
//     (grad psi_i: transform of the coefficients i G c_i(G), exact for the
//     plane-wave expansion); every sum over orbitals in double
//   candidates: rho > <rho> and |grad rho| < <|grad rho|>, ascending grid index
//   pivots: column-pivoted QR of Psi^* on the candidate columns, as Gram-Schmidt
//     with re-orthogonalisation: at step k the column of largest residual norm
//     (ties to the lowest index), residual norms downdated by (q_k . a_j)^2
//   Phi = (V V^T)^{-1/2} V Psi, V[k][i] = psi_i(r_{C_k}): the polar factor of V
//     by the Newton-Schulz iteration X <- X (3 I - X^T X) / 2 from V / |V|_F
// All of it in double; the orbitals' real-space values come in the plan's
// precision.
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
        double s = 0;
        if (dphi) {
            for (int i = 0; i < n; ++i) s += (double)phi[i * N + r] * (double)dphi[i * N + r];
            out[r] = 2.0 * s;
        } else {
            for (int i = 0; i < n; ++i) {
                const double v = (double)phi[i * N + r];
                s += v * v;
            }
            out[r] = s;
        }
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

// A[i][s] = phi_i(r_s) in double, r_s = sel[s] (sel == nullptr: r_s = s)
template <typename R>
__global__ void gather_columns_kernel(const R* __restrict__ phi, long long N, const int* __restrict__ sel,
                                      long long m, double* __restrict__ A) {
    const int i = blockIdx.y;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < m; s += (long long)gridDim.x * blockDim.x)
        A[i * m + s] = (double)phi[i * N + (sel ? sel[s] : s)];
}

// ------------------------------------------------------ column-pivoted QR

// nu[j] = |a_j|^2 and the block's largest
__global__ void qr_init_kernel(const double* __restrict__ A, int n, long long m, double* __restrict__ nu,
                               ArgMax* __restrict__ part) {
    ArgMax best{-1.0, -1};
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
        double s = 0;
        for (int i = 0; i < n; ++i) {
            const double v = A[i * m + j];
            s += v * v;
        }
        nu[j] = s;
        best = better(best, ArgMax{s, j});
    }
    best = block_argmax(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// nu[j] -= (q_k . a_j)^2 for the columns not chosen yet (nu < 0 marks chosen
// ones), and the block's largest
__global__ void qr_update_kernel(const double* __restrict__ A, int n, long long m, const double* __restrict__ qk,
                                 double* __restrict__ nu, ArgMax* __restrict__ part) {
    extern __shared__ double q[];
    for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] = qk[i];
    __syncthreads();
    ArgMax best{-1.0, -1};
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
        double v = nu[j];
        if (v < 0) continue;
        double d = 0;
        for (int i = 0; i < n; ++i) d += q[i] * A[i * m + j];
        v -= d * d;
        if (v < 0) v = 0;
        nu[j] = v;
        best = better(best, ArgMax{v, j});
    }
    best = block_argmax(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

// One block: the pivot of step k from the block partials; q_k = the
// normalised residual of its column against q_0..q_{k-1} (two Gram-Schmidt
// passes).  status = 1 when the largest residual norm^2 is not above 1e-10
// times the largest column norm^2 (kept in *nu0 at step 0): the candidate
// columns do not span n_occ dimensions beyond rounding.
__global__ void qr_pick_kernel(const ArgMax* __restrict__ part, int nparts, const double* __restrict__ A, int n,
                               long long m, double* __restrict__ Q, int k, int* __restrict__ piv,
                               double* __restrict__ nu, double* __restrict__ nu0, int* __restrict__ status) {
    extern __shared__ double sh[];
    double* r = sh;      // n
    double* c = sh + n;  // k coefficients
    __shared__ long long s_p;
    __shared__ double s_norm;
    ArgMax best{-1.0, -1};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) best = better(best, part[b]);
    best = block_argmax(best);
    if (threadIdx.x == 0) {
        if (k == 0) *nu0 = best.v;
        const bool ok = best.j >= 0 && best.v > 1e-10 * *nu0 && best.v == best.v;
        s_p = ok ? best.j : -1;
        if (!ok) *status = 1;
        if (ok) {
            piv[k] = (int)best.j;
            nu[best.j] = -1.0;
        }
    }
    __syncthreads();
    if (s_p < 0) return;
    for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] = A[i * m + s_p];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        for (int l = threadIdx.x; l < k; l += blockDim.x) {
            double s = 0;
            for (int i = 0; i < n; ++i) s += Q[(long long)l * n + i] * r[i];
            c[l] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double s = r[i];
            for (int l = 0; l < k; ++l) s -= c[l] * Q[(long long)l * n + i];
            r[i] = s;
        }
        __syncthreads();
    }
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += r[i] * r[i];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        s_norm = sqrt(s);
        if (!(s > 0)) *status = 1;
    }
    __syncthreads();
    if (!(s_norm > 0)) return;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Q[(long long)k * n + i] = r[i] / s_norm;
}

// grid point of each pivot column: out[k] = sel[piv[k]] (sel null: piv[k])
__global__ void map_pivots_kernel(const int* __restrict__ piv, const int* __restrict__ sel, int n,
                                  int* __restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        out[k] = sel ? sel[piv[k]] : piv[k];
}

// ------------------------------------------------------ polar factor

// X[k][i] = A[i][piv[k]] / |V|_F (one block)
__global__ void polar_start_kernel(const double* __restrict__ A, int n, long long m, const int* __restrict__ piv,
                                   double* __restrict__ X) {
    __shared__ double s_inv;
    double s = 0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int k = e / n, i = e - k * n;
        const double v = A[(long long)i * m + piv[k]];
        X[e] = v;
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) s_inv = 1.0 / sqrt(s);
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) X[e] *= s_inv;
}

// C = A op(B), n x n, op(B) = B^T when trans_b; 16 x 16 tiles
__global__ void dgemm_small_kernel(const double* __restrict__ A, const double* __restrict__ B, int n, int trans_b,
                                   double* __restrict__ C) {
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
    if (row < n && col < n) C[(long long)row * n + col] = s;
}

// err[0] = max |T - I| (one block)
__global__ void orth_error_kernel(const double* __restrict__ T, int n, double* __restrict__ err) {
    __shared__ double s[kThreads];
    double e = 0;
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) {
        const int i = k / n, j = k - i * n;
        e = fmax(e, fabs(T[k] - (i == j ? 1.0 : 0.0)));
    }
    s[threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) err[0] = s[0];
}

// X <- 1.5 X - 0.5 Y
__global__ void ns_combine_kernel(double* __restrict__ X, const double* __restrict__ Y, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        X[e] = 1.5 * X[e] - 0.5 * Y[e];
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
cudaError_t launch_gather_columns(const R* phi, int n, long long N, const int* sel, long long m, double* A,
                                  cudaStream_t st) {
    dim3 grid((unsigned)std::min<long long>((m + kThreads - 1) / kThreads, 1024), (unsigned)n);
    gather_columns_kernel<R><<<grid, kThreads, 0, st>>>(phi, N, sel, m, A);
    return cudaGetLastError();
}

int scdm_qr_blocks(long long m) {
    const long long b = (m + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));  // 8 blocks of 256 per SM at most
}

size_t scdm_argmax_bytes() { return sizeof(ArgMax); }

cudaError_t launch_qr_init(const double* A, int n, long long m, double* nu, void* part, cudaStream_t st) {
    qr_init_kernel<<<scdm_qr_blocks(m), kThreads, 0, st>>>(A, n, m, nu, (ArgMax*)part);
    return cudaGetLastError();
}

cudaError_t launch_qr_update(const double* A, int n, long long m, const double* qk, double* nu, void* part,
                             cudaStream_t st) {
    qr_update_kernel<<<scdm_qr_blocks(m), kThreads, n * sizeof(double), st>>>(A, n, m, qk, nu, (ArgMax*)part);
    return cudaGetLastError();
}

cudaError_t launch_qr_pick(const void* part, long long m, const double* A, int n, double* Q, int k, int* piv,
                           double* nu, double* nu0, int* status, cudaStream_t st) {
    qr_pick_kernel<<<1, kThreads, (size_t)(n + k + 1) * sizeof(double), st>>>(
        (const ArgMax*)part, scdm_qr_blocks(m), A, n, m, Q, k, piv, nu, nu0, status);
    return cudaGetLastError();
}

cudaError_t launch_map_pivots(const int* piv, const int* sel, int n, int* out, cudaStream_t st) {
    map_pivots_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(piv, sel, n, out);
    return cudaGetLastError();
}

cudaError_t launch_polar_start(const double* A, int n, long long m, const int* piv, double* X, cudaStream_t st) {
    polar_start_kernel<<<1, kThreads, 0, st>>>(A, n, m, piv, X);
    return cudaGetLastError();
}

// One Newton-Schulz step X <- X (3 I - X^T X) / 2 written as 1.5 X - 0.5 (X X^T) X
// (the same map for the polar factor of a square X); err[0] = max |X X^T - I|
// before the step.
cudaError_t launch_newton_schulz_step(double* X, double* T, double* Y, int n, double* err, cudaStream_t st) {
    dim3 g((n + 15) / 16, (n + 15) / 16);
    dgemm_small_kernel<<<g, 256, 0, st>>>(X, X, n, 1, T);
    orth_error_kernel<<<1, kThreads, 0, st>>>(T, n, err);
    dgemm_small_kernel<<<g, 256, 0, st>>>(T, X, n, 0, Y);
    ns_combine_kernel<<<grid_for((long long)n * n), kThreads, 0, st>>>(X, Y, (long long)n * n);
    return cudaGetLastError();
}

template cudaError_t launch_deriv_coeffs<float>(const cx<float>*, int, int, const double*, cx<float>*, cudaStream_t);
template cudaError_t launch_deriv_coeffs<double>(const cx<double>*, int, int, const double*, cx<double>*,
                                                 cudaStream_t);
template cudaError_t launch_orbital_sum<float>(const float*, const float*, int, long long, double*, cudaStream_t);
template cudaError_t launch_orbital_sum<double>(const double*, const double*, int, long long, double*, cudaStream_t);
template cudaError_t launch_gather_columns<float>(const float*, int, long long, const int*, long long, double*,
                                                  cudaStream_t);
template cudaError_t launch_gather_columns<double>(const double*, int, long long, const int*, long long, double*,
                                                   cudaStream_t);

}  // namespace ace
