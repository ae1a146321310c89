// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace ace {

// Prologue: how a pass fills its shared-memory tile.
enum Prologue {
    PRO_LOAD = 0,   // complex source box of transform t
    PRO_PAIR = 1,   // f_a phi_b + i f_c phi_d (two pair densities, Eq. 3)
    PRO_PACK2 = 2,  // f_a + i f_c (two real functions in one complex transform)
};
// Epilogue: where the transformed tile goes.
enum Epilogue {
    EPI_STORE = 0,  // complex destination box of transform t
    EPI_SPLIT = 1,  // real part -> out[a], imaginary part -> out[c], times scale
    EPI_ACCUM = 2,  // exchange accumulation W_a += v phi_b (and W_b += v f_a), pair energies
};
// What happens between the transforms of the z axis.
enum Middle {
    MID_NONE = 0,
    MID_COULOMB = 1,  // forward z, times 4 pi / |G|^2 / N (G = 0 -> 0), inverse z
};

// Quadruple of function indices for one packed transform: (a, b) and (c, d);
// c < 0 when the imaginary half is empty.
struct Quad {
    int a, b, c, d;
};

struct PassArgs {
    int n0, n1, n2;  // box extents (z, y, x); x is contiguous
    int tz, ty, tx;  // tile extents (divide the box extents)
    int axes;        // 1 = x, 2 = y (needs tz == 1), 4 = z
    int bulk;        // spectrum tiles by bulk async copies (16-byte aligned runs)
    int vec;         // real functions as 4-wide vectors (tx, n2 multiples of 4)
    int* err;        // device error flag (1: a bounded wait timed out)
    int lookahead;   // transforms ahead whose inputs a block pulls into L2 (0: none)
    AxisPlan px, py, pz;
    const void *twx, *twy, *twz;  // exp(-2 pi i j / n) per axis, cx<R>
    // prologue
    const void* src;
    long long src_tstride;  // elements between transforms
    const void* fl;         // left functions  [*][N] real
    const void* fr;         // right functions [*][N] real
    const Quad* quads;      // per transform (indexed from t0)
    int t0;
    // epilogue
    void* dst;
    long long dst_tstride;
    void* accl;  // EPI_SPLIT: real outputs; EPI_ACCUM: left accumulators
    void* accr;  // EPI_ACCUM: right accumulators (symmetric mode)
    int symmetric;
    double* e_part;  // EPI_ACCUM: [transform][tile][2]
    double scale;    // EPI_SPLIT output scale
    // Coulomb kernel
    double b[9];  // reciprocal vectors as rows
    double kscale;
    const int* freq[3];  // per axis: frequency held at each position after the forward stages
    const void* kern;    // per-pencil Coulomb pass: 4 pi / |G|^2 / N in spectrum layout, [n0][n1][n2] float
    int kern_inline;     // 1: the tile passes' Coulomb stage reads K(G) / N from kern ([n0][n1][n2], type R,
                         // by x slot) instead of forming 4 pi / |G|^2 (cut-off interaction; double precision)
    int r0;              // compile-time cube kernels: first radix of every axis (0: make_axis_plan's plan);
                         // nonzero only for the pair passes, with freq and kern made for that plan
};

struct PassShape {
    int tz, ty, tx, axes, threads, bulk, vec;
    int cube;  // 1: use the compile-time kernel of this N^3 box (single precision)
    size_t smem;
};

// N^3 boxes with compile-time pass kernels, and their tile geometry (shared by
// the host planner and the kernel instantiations).
constexpr bool cube_supported(int n) {
    return n == 32 || n == 60 || n == 80 || n == 90 || n == 96 || n == 100 || n == 108 || n == 120 || n == 160;
}
// threads of a plane block: the butterfly counts of both stages divide evenly
constexpr int cube_xy_threads(int n) {
    return n == 32 ? 128 : n == 96 ? 256 : n == 120 ? 480 : n == 160 ? 320 : (n * n >= 12000 ? 512 : 256);
}
// Plane layout of N % 16 == 0 cubes: within each 16-element block of a row,
// x position p sits in slot p ^ w, w = (((p >> 4) + s_N y) & 7) | ((y & 1) << 3);
// the permutation is its own inverse and keeps blocks in place.  Bit 3 of w
// alternates bank halves between neighbouring rows (the strided x stage: two
// rows per half-warp, 8 butterflies each); the low bits rotate with the row by
// s_N so that the contiguous x stage, whose 16 butterflies per half-warp run
// across a row boundary (12 per row at N = 96), lands on 16 distinct 8-byte
// bank pairs: s_N = 6 at N = 96 (radix 8 last), 5 at 80, 2 at 32, by a count
// of the bank conflicts of every stage's accesses for each s in 0..7 (at 160
// no s helps by more than 1%).  Columns always read 16 consecutive slots.
constexpr bool cube_swizzle(int n) { return n % 16 == 0; }
__host__ __device__ constexpr int plane_swizzle_rot(int n) { return n == 96 ? 6 : n == 80 ? 5 : n == 32 ? 2 : 0; }
__host__ __device__ constexpr int plane_swizzle(int p, int y, int n) {
    return p ^ ((((p >> 4) + plane_swizzle_rot(n) * y) & 7) | ((y & 1) << 3));
}
constexpr int cube_z_threads(int) { return 256; }
constexpr int cube_z_tx(int n) {  // largest even divisor of n up to 32
    for (int d = 32; d >= 2; d -= 2)
        if (n % d == 0) return d;
    return 1;
}
constexpr int cube_z_ty(int n) {  // largest divisor keeping the tile within 8192 elements
    for (int d = n; d >= 1; --d)
        if (n % d == 0 && n * d * cube_z_tx(n) <= 8192) return d;
    return 1;
}

// Pencils per warp of the per-pencil Coulomb pass (zline.cuh): the largest
// even divisor of n^2 up to 16 (even: a z row of the group is a whole number
// of 16-byte units).
constexpr int zline_group(int n) {
    for (int g = 16; g >= 2; g -= 2)
        if ((n * n) % g == 0) return g;
    return 0;
}
cudaError_t zline_coulomb_launch(int n, const PassArgs& a, int batch, cudaStream_t st);
// First radices, besides make_axis_plan's, of the two-stage plans the pair
// passes have compile-time kernels for on an n^3 box (the autotuner times
// them): written to r0[], count returned (at most 3).
inline int pair_radix_alternatives(int n, int* r0) {
    switch (n) {
        case 96: r0[0] = 8; r0[1] = 16; return 2;    // 8 x 12, 16 x 6 (default 12 x 8)
        case 120: r0[0] = 10; r0[1] = 8; return 2;   // 10 x 12, 8 x 15 (default 12 x 10)
        case 160: r0[0] = 10; return 1;              // 10 x 16 (default 16 x 10)
        default: return 0;
    }
}
// plane passes with transposed spectrum planes (plane.cuh), N^3 boxes with
// N % 8 == 0: which = 0 pair product + forward, 1 inverse + exchange accumulation
constexpr bool tplane_supported(int n) { return n % 8 == 0; }
// ... and as one persistent kernel (its pencil groups: 16 per warp, N / 16 warps)
constexpr bool pipeline_supported(int n) { return n % 16 == 0; }
cudaError_t tplane_pair_launch(int n, int which, const PassArgs& a, int batch, cudaStream_t st);
// plane passes on clusters of two half-plane blocks (halfplane.cuh): which =
// 0 pair product + forward, 1 inverse + exchange accumulation; n = 120
constexpr bool halfplane_supported(int n) { return n == 120; }
cudaError_t halfplane_pair_launch(int n, int which, const PassArgs& a, int batch, cudaStream_t st);
// the three pair passes as one persistent kernel (pipeline.cuh), same boxes
struct PipeArgs {
    int ntrans;       // packed transforms: quads a.t0 .. a.t0 + ntrans - 1
    int lag;          // steps between a transform's passes
    int slots;        // spectrum ring (transforms), PassArgs::dst
    int* done;        // [3][ntrans] finished items per pass and transform
    int* ticket;      // next item
    int* abort_flag;  // set by a timed-out wait
    int discard;      // drop dead spectrum planes from L2 unwritten
    int prefetch;     // fetch tickets two items ahead
};
cudaError_t pipeline_pair_launch(int n, const PassArgs& a, const PipeArgs& p, cudaStream_t st);

#if defined(__CUDACC__)
// Sum of v over the 32 lanes of a warp in float-float arithmetic (Knuth's
// TwoSum at every step, the rounding error carried in lo): about 2^-44 of
// the sum of |v| on the FP32 pipes, where a double reduction would queue on
// this GPU's FP64 pipe (a small fraction of the FP32 rate).  Every lane gets
// the same result (TwoSum's error is exact, so both orders of a step agree).
__device__ __forceinline__ double warp_sum_ff(float v) {
    float hi = v, lo = 0.0f;
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = hi + h2, bp = s - hi;
        const float err = (hi - (s - bp)) + (h2 - bp);
        hi = s;
        lo = lo + l2 + err;
    }
    return (double)hi + (double)lo;
}
#endif

// True while `st` records into a CUDA graph: launchers then leave kernel
// attributes alone (set by the same launch outside capture before).
inline bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// compile-time cube passes (cube_*.cu), single precision
cudaError_t cube_pass_launch(int n, const PassArgs& a, const PassShape& s, int pro, int epi, int mid, int sgn,
                             int batch, cudaStream_t st);

// Launch one pass over `batch` transforms (gridDim.y) of the box.
template <typename R>
cudaError_t launch_pass(const PassArgs& a, const PassShape& s, int pro, int epi, int mid, int sgn, int batch,
                        cudaStream_t st);


// ---------------------------------------------------------- other kernels

// box[t] (zeroed by the caller) <- c_a(G) + i c_b(G) at +G, conj at -G
// (idx_pos / idx_neg: box positions of +G / -G in digit-reversed order).
template <typename R>
cudaError_t launch_scatter(const cx<R>* psi, const Quad* quads, int t0, int batch, int npw, const int* idx_pos,
                           const int* idx_neg, cx<R>* box, long long N, cudaStream_t st);
// out_a(G) = s (Z(G) + Z(-G)^*) / 2, out_c(G) = s (Z(G) - Z(-G)^*) / (2i) on the half sphere.
template <typename R>
cudaError_t launch_gather(const cx<R>* box, const Quad* quads, int t0, int batch, int npw, const int* idx_pos,
                          const int* idx_neg, long long N, double s, cx<R>* out, cudaStream_t st);

// Partial Gamma Gram products: P[chunk][i][j] = sum_{k in chunk} A[i][k] B[j][k]
// over the real views A [m][K], B [n][K] (K = 2 n_pw_half), double partials.
template <typename R>
cudaError_t launch_gram_partial(const R* A, const R* B, int m, int n, long long K, int nchunk, double* P,
                                cudaStream_t st);
// The same partials on tcgen05 tensor cores, streamed (umma_stream.cu): split
// TF32, FP32 accumulation in TMEM, P [ceil(K / kchunk)][m][n] float; kchunk a
// multiple of 32 from gram_stream_kchunk (about one block per SM, at most
// max_k reals per slice when max_k > 0); err: device error flag for bounded waits.
long long gram_stream_kchunk(int m, int n, long long K, int sms, int max_k);
// absval: products of |A| and |B| (the overlap integrals of the s-MTACE screen).
cudaError_t launch_gram_stream(const float* A, const float* B, int m, int n, long long K, long long kchunk, float* P,
                               int* err, cudaStream_t st, bool absval = false);
// out[t][j] = -sum_k C[t][k] xi[k][j] on tcgen05 (K psi = -xi C^T, Eq. 5):
// C [T][n] double, xi [n][K] float, out [T][K] float; Cimg: scratch of
// apply_product_scratch(T, n) floats (16-byte aligned) for C's TF32 split.
// Ximg (or null): xi's split image from launch_xi_image, which feeds xi to the
// tensor cores by bulk copies instead of the producer warps.
size_t apply_product_scratch(int T, int n);
cudaError_t launch_apply_product(const double* C, int T, int n, const float* xi, long long K, float* Cimg, float* out,
                                 int sms, int* err, cudaStream_t st, const float* Ximg = nullptr);
// xi [n][K] float -> Ximg: xi_image_floats(n, K) floats (16-byte aligned), the
// TF32 hi / lo split of xi^T in the product's swizzled operand tiles.
size_t xi_image_floats(int n, long long K);
cudaError_t launch_xi_image(const float* xi, int n, long long K, float* Ximg, cudaStream_t st);
// The same on CUDA cores with double partials over nchunk K-slices.
template <typename R>
cudaError_t launch_overlap_partial(const R* A, int m, long long K, int nchunk, double* P, cudaStream_t st);
// G [m][m] = scale * sum over the slices of the partials.
template <typename PT>
cudaError_t launch_overlap_finish(const PT* P, int nchunk, int m, double scale, double* G, cudaStream_t st);
// launch_gram_finish for single-precision partials
cudaError_t launch_gram_finish_f32(const float* P, int nchunk, const float* A, const float* B, int m, int n,
                                   long long K, double* G, int ldg, cudaStream_t st);
// G[i][j] = 2 sum_c P[c][i][j] - (A_i0 B_j0 + A_i1 B_j1)   (G = 0 counted once)
template <typename R>
cudaError_t launch_gram_finish(const double* P, int nchunk, const R* A, const R* B, int m, int n, long long K,
                               double* G, int ldg, cudaStream_t st);

// out[i][c] = alpha sum_k A[i][k] B[k][c]  (A double [m][k], B R [k][ncols], out R);
// fp64_math: products and sums in double, else in R over 16-wide slices with
// compensated slice accumulation; lower: A is lower triangular (k <= row).
template <typename R>
cudaError_t launch_gemm_nn(const double* A, int m, int k, const R* B, long long ncols, double alpha, R* out,
                           bool fp64_math, cudaStream_t st, bool lower = false);

// ---- SCDM localisation (Sections 2.4-2.5; scdm.cu), every result in double
// out[i][p] = i gd[p] psi[i][p] (the coefficients of d psi_i / d r_d)
template <typename R>
cudaError_t launch_deriv_coeffs(const cx<R>* psi, int n, int npw, const double* gd, cx<R>* out, cudaStream_t st);
// out[r] = sum_i phi_i(r)^2 (dphi null) or 2 sum_i phi_i(r) dphi_i(r); phi, dphi [n][N]
template <typename R>
cudaError_t launch_orbital_sum(const R* phi, const R* dphi, int n, long long N, double* out, cudaStream_t st);
// means[0] = <rho>, means[1] = <|grad rho|> (grad [3][N]); part: 2 scdm_stats_blocks(N) doubles
int scdm_stats_blocks(long long N);
cudaError_t launch_scdm_stats(const double* rho, const double* grad, long long N, double* part, double* means,
                              cudaStream_t st);
// sel <- ascending grid points with rho > means[0] and |grad rho| < means[1];
// counts [scdm_select_blocks(N)], offsets [scdm_select_blocks(N) + 1] (the last: how many)
int scdm_select_blocks(long long N);
cudaError_t launch_scdm_select(const double* rho, const double* grad, long long N, const double* means, int* counts,
                               int* offsets, int* sel, cudaStream_t st);
// A[i][s] = phi_i(r_s), r_s = sel[s] (sel null: s), A [n][m] in the orbitals' precision
template <typename R>
cudaError_t launch_gather_columns(const R* phi, int n, long long N, const int* sel, long long m, R* A,
                                  cudaStream_t st);
// Column-pivoted QR of A [n][m] by Gram-Schmidt applied twice, all products in
// double: launch_qr_init, then launch_qr_step for k = 0 .. n-1 (step k picks
// pivot k and, below n - 1, updates the residual norms).  part:
// scdm_qr_blocks(m) argmax partials of scdm_argmax_bytes() each; nu [m]
// residual norms; R [n][m] coefficients q_l . a_j; Q [n][n] (row k = q_k);
// r, c [n] scratch; piv [n] columns of A; nu0 one double; status set to 1 on
// rank deficiency (a best residual norm^2 not above 1e-10 of the largest
// column norm^2).
int scdm_qr_blocks(long long m, int n, int esz);  // esz: bytes of an element of A
size_t scdm_argmax_bytes();
struct QrWork {
    void* part;
    double *nu, *R, *Q, *r, *c, *nu0, *rdiag;  // rdiag [n]: R[k][k] = |r_k|
    int *piv, *status;
};
template <typename T>
cudaError_t launch_qr_init(const T* A, int n, long long m, double* nu, void* part, cudaStream_t st);
template <typename T>
cudaError_t launch_qr_step(const T* A, int n, long long m, int k, QrWork w, cudaStream_t st);
// out[k] = sel[piv[k]] (sel null: piv[k]): the pivots' grid points
cudaError_t launch_map_pivots(const int* piv, const int* sel, int n, int* out, cudaStream_t st);
// X [n][n] = V / |V|_F, V[k][i] = A[i][piv[k]], fro = |V|_F; one Newton-Schulz
// step toward its polar factor with the scaling alpha (Chen & Chow, SIAM J.
// Matrix Anal. Appl. 35 (2014)), T, Y [n][n] scratch, err[0] = max |X X^T - I|
// before it
template <typename T>
cudaError_t launch_polar_start(const T* A, int n, long long m, const int* piv, double* X, double* fro,
                               cudaStream_t st);
cudaError_t launch_newton_schulz_step(double* X, double* T, double* Y, int n, double alpha, double* err,
                                      cudaStream_t st);

// The same product with A double, B and out float in float-float arithmetic
// (about 2^-44 of sum |A||B|) on the FP32 pipes.
cudaError_t launch_gemm_nn_ff(const double* A, int m, int k, const float* B, long long ncols, double alpha, float* out,
                              bool lower, cudaStream_t st);

// The same over many thread blocks (blocked right-looking factorisation and
// column-block inverse): work holds neg_cholesky_work(n) doubles; *nlaunch
// receives the number of kernels launched.
size_t neg_cholesky_work(int n);
cudaError_t launch_neg_cholesky_blocked(const double* M, int n, double* L, double* Linv, int* status, double* work,
                                        int* nlaunch, cudaStream_t st);

// Cholesky of -M and the inverse of its factor, in double, one thread block.
// status: 0 ok, 1 not positive definite.
cudaError_t launch_neg_cholesky_inverse(const double* M, int n, double* L, double* Linv, int* status,
                                        cudaStream_t st);

// E[0] = coef * sum_t sum_tile (w1 e1 + w2 e2), deterministic order; E[1 ..]
// holds up to 16384 block sums (room for 1 + 16384 doubles).
cudaError_t launch_energy_reduce(const double* e_part, const Quad* quads, int ntrans, int ntiles, double coef,
                                 double* E, cudaStream_t st);

// out[0] = coef * sum_k x[k]^2 (one block, fixed order)
cudaError_t launch_sumsq(const double* x, long long n, double coef, double* out, cudaStream_t st);

// One block waiting up to limit_ms on a barrier nothing completes; sets *err.
cudaError_t launch_wait_for_nothing(int* err, int limit_ms, cudaStream_t st);

// Record an ACE_ERR_* code and message for ace_last_error(); returns code.
int set_last_error(int code, const char* msg);

}  // namespace ace
