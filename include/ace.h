/*
 * ace.h -- C ABI of the GB300 library that builds and applies the adaptively
 * compressed exchange (ACE) operator, the data-parallel hot path of the
 * MTACE / s-MTACE schemes of arXiv:2110.07670 (Mandal, Kar, Kloeffel, Meyer,
 * Nair).
 *
 * What the calls compute (Section 2.1-2.2 of the paper, Eq. 1-5):
 *   V_X phi_i   = -sum_j v_ij(r) phi_j(r)                         (Eq. 2)
 *   v_ij(r)     = <phi_j| 1/r12 |phi_i>, solved in reciprocal space  (Eq. 3)
 *   E_X         = -sum_{i,j} <phi_i| v_ij |phi_j>                  (Eq. 4)
 *   V_X^ACE     = -sum_k |P_k><P_k|                                (Section 2.2)
 *   V_X^ACE psi = -sum_k P_k <P_k|psi>                             (Eq. 5)
 * with every exchange quantity scaled by the exact-exchange fraction alpha
 * (PBE0: 0.25).  The ACE vectors are xi = P = W L^-T, where W = alpha V_X Phi,
 * M = Phi^T W and -M = L L^T; the operator K = -xi xi^T equals alpha V_X on
 * the span of the occupied orbitals.
 *
 * Conventions (all arrays row-major, C order):
 *  - cell[9]: lattice vectors a1, a2, a3 as rows, bohr.  Reciprocal vectors
 *    b = 2 pi inv(A)^T.  G = h b1 + k b2 + l b3.
 *  - Plane waves: |G|^2 <= ecut_ry (bohr^-2; Ry units make |G|^2 the kinetic
 *    energy), the convention that reproduces the plane-wave counts of the
 *    paper's Table 1.
 *  - Gamma point: orbitals are real, c(-G) = c(G)^*, and only the half sphere
 *    {h>0} U {h=0,k>0} U {h=k=0,l>=0} is stored, in lexicographic (h,k,l)
 *    order (G = 0 is entry 0).  n_pw_half entries per vector.  Im c(0) must be
 *    zero (|Im c(0)| > 1e-6 is ACE_ERR_INVALID_ARG).
 *  - psi(r) = Omega^-1/2 sum_G c(G) e^{iG.r}; a normalised orbital has full-
 *    sphere sum |c|^2 = 1.
 *  - Real-space grid grid[3] = (n0, n1, n2) along (a1, a2, a3); each n is a
 *    product of 2, 3, 5 and n_d >= 2 max|Miller_d| + 1.
 *  - Coulomb kernel 4 pi / |G|^2 on every G of the FFT box (folded to
 *    -n/2..n/2-1), G = 0 term dropped; or the interaction cut off at a radius
 *    (ace_opts.coulomb_rc), or the G = 0 term from the auxiliary-function
 *    correction (ace_opts.coulomb_g0).
 *  - Vectors are complex, interleaved (re, im): complex128 for ACE_FP64 plans,
 *    complex64 for ACE_MIXED plans.  [rows][n_pw_half].
 *
 * Ownership: every vector argument is a DEVICE pointer owned by the caller;
 * pair lists and E_x are HOST pointers.  The library owns only the plan (its
 * workspace, FFT plans and device-side pair lists), created and destroyed
 * explicitly.  Work is enqueued on the given CUDA stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream); calls that return a host
 * scalar (E_x) synchronise that stream.  A plan may be used by one host
 * thread at a time.
 *
 * Errors: every call returns ACE_OK (0) or a negative code; ace_last_error()
 * gives the message of the calling thread's last failure.
 */
#ifndef ACE_H
#define ACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ACE_OK = 0,
    ACE_ERR_INVALID_ARG = -1,
    ACE_ERR_GRID_TOO_SMALL = -2, /* n_d < 2 max|Miller_d| + 1, or a prime factor above 5 */
    ACE_ERR_NOT_POSDEF = -3,     /* -M is not positive definite (dependent or zero orbitals) */
    ACE_ERR_OOM = -4,
    ACE_ERR_CUDA = -5,
    ACE_ERR_TIMEOUT = -6 /* a bounded device-side wait gave up */
};

enum { ACE_FP64 = 0, ACE_MIXED = 1 };

typedef struct ace_plan ace_plan;

typedef struct {
    int pair_batch;    /* packed pair transforms per pass launch; 0 = automatic */
    int kernels;       /* 0: fastest available; 1: CUDA-core Gram products instead of
                          tcgen05 tensor cores; 2: also generic (runtime-size) FFT passes */
    int pair_streams;  /* streams the pair sub-batches overlap on; 0 = automatic,
                          1 = every pass in order on the call's stream */
    int pair_variant;  /* kernels of the pair passes (Eq. 2-4): 1 tile passes, 2 transposed-
                          plane passes, 3 one persistent kernel for all three passes, 4 the
                          plane-kernel forward pass with the tile passes after it, 5 the
                          plane passes on clusters of two blocks holding half a plane each
                          (2: single precision, n^3 boxes with n in {32, 80, 96, 120, 160};
                          3: single precision, n in {32, 80, 96, 160};
                          4: single precision, n in {32, 60, 80, 90, 96, 100, 108, 120, 160};
                          5: single precision, n = 120);
                          0 = automatic: where several apply (and pair_streams is 0, both 1
                          and 2 streams) they are timed at plan creation on the plan's own
                          buffers and the fastest is kept (see ace_plan_config) */
    double coulomb_rc; /* G = 0 treatment of the Poisson solve (Eq. 3): 0 = the bare
                          4 pi / |G|^2 with the G = 0 term dropped (neutralising
                          background); > 0 = the interaction 1/r cut off at r = coulomb_rc
                          bohr (Spencer & Alavi, Phys. Rev. B 77, 193110 (2008)):
                          4 pi (1 - cos(|G| R_c)) / |G|^2, and 2 pi R_c^2 at G = 0; the
                          usual choice is R_c = (3 Omega / 4 pi)^(1/3).  Negative or
                          non-finite: ACE_ERR_INVALID_ARG.  Applies to every build and to
                          hfx_apply_exact of the plan. */
    int coulomb_g0;    /* with coulomb_rc = 0: 1 = keep the bare kernel's G = 0 term as
                          K(0) = 4 pi chi, the auxiliary-function correction for Gamma-only
                          sampling (Gygi & Baldereschi, Phys. Rev. B 34, 4405 (1986)),
                          chi = Omega / (2 pi)^3 int F d^3q - sum_{G != 0} F(G) + alpha for
                          F(q) = exp(-alpha q^2) / q^2 over the whole reciprocal lattice
                          (independent of alpha; for a cubic cell K(0) / Omega = xi_M / L,
                          the Madelung term); 0 = drop it.  1 with coulomb_rc > 0, or any
                          other value: ACE_ERR_INVALID_ARG. */
} ace_opts;

/*
 * Create a plan for one system: grid, cell, cutoff, the largest occupied set
 * it will see, and the precision (ACE_FP64: every step in double; ACE_MIXED:
 * FFTs, pair products and W in float, M / Cholesky / triangular solve / E_x
 * in double).  opts may be NULL.  Allocates the plan's device workspace on the
 * current device.
 */
int ace_plan_create(ace_plan** plan, const int grid[3], const double cell[9], double ecut_ry, int n_occ_max,
                    int precision, const ace_opts* opts);

void ace_plan_destroy(ace_plan* plan);

/* The plan's pair-pass kernels: pair_variant (1 to 5 as in ace_opts),
 * pair_streams, and, where plan creation timed them, tune_ms[6] = ms per
 * timing run of {tile passes on 1 stream, on 2 streams, transposed-plane
 * passes, persistent kernel, hybrid, half-plane pairs} (0 = not timed).  Any
 * output may be NULL. */
int ace_plan_config(const ace_plan* plan, int* pair_variant, int* pair_streams, float* tune_ms);

/* The pair-tile shape of the plan's pair passes: row_block = 0 packs
 * consecutive pairs of the row-ordered list two per transform; 2, 4 or 8
 * packs (i1, j) with (i2, j) -- pairs sharing their column orbital -- in
 * blocks of that many rows, so one fresh orbital and one merged accumulator
 * update serve each transform while the block's rows stay in L2.  Plan
 * creation times the four at the chosen pair_variant (row_block_ms[4], 0 =
 * not timed) unless the environment fixes ACE_ROW_BLOCK.  With ACE_TUNE_CACHE
 * naming a file, the choice of pair_variant, pair_streams and row_block is
 * looked up there by grid, n_occ_max, precision and device before any timing
 * and appended after it (*from_cache = 1 when it came from the file).  Any
 * output may be NULL. */
int ace_plan_tuning(const ace_plan* plan, int* row_block, float* row_block_ms, int* from_cache);

/* The radix plan of the pair passes' 3D FFTs (the Poisson solves of Eq. 3):
 * every axis of the box in two stages, radix *radix0 and then n / *radix0.
 * On single-precision n^3 plans with n = 96, 120 or 160, plan creation times
 * each candidate plan (96: 12 x 8, 8 x 12, 16 x 6; 120: 12 x 10, 10 x 12,
 * 8 x 15; 160: 16 x 10, 10 x 16) with every pair_variant and keeps the
 * fastest: candidates[k] are their first radices, candidate_ms[k] the best
 * pair-pass time of each (k < *n_candidates <= 4; later entries 0).  Other
 * plans have one candidate, make_axis_plan's.  The pair passes' spectrum
 * never leaves them, so the orbital and W transforms keep the first
 * candidate's plan.  ACE_PAIR_RADIX=<first radix> in the environment fixes the
 * plan (a radix that is no candidate of the grid: ACE_ERR_INVALID_ARG at plan
 * creation); ACE_TUNE_CACHE lines carry the choice.  Any output may be NULL. */
int ace_plan_radix(const ace_plan* plan, int* radix0, int* n_candidates, int* candidates, float* candidate_ms);

/* Number of half-sphere plane waves and, when miller != NULL, their Miller
 * indices [n_pw_half][3] (host memory, canonical order). */
int ace_gvec(const ace_plan* plan, int* n_pw_half, int32_t* miller);

/*
 * Build the ACE operator (an outer MTS step, Section 2.3): every listed pair
 * density phi_i phi_j, its Poisson solve (Eq. 3), W = alpha V_X Phi (Eq. 2),
 * M = Phi^T W, -M = L L^T, xi = W L^-T, and E_x = -alpha sum (2 - d_ij) e_ij
 * over the listed pairs i <= j (Eq. 4).
 *   psi_G  [n_occ][n_pw_half] device, orthonormal occupied orbitals
 *   pair_row_ptr[n_occ+1], pair_col[]: host CSR of the kept pairs (row i lists
 *          columns j >= i, ascending); both NULL = every pair i <= j
 *   xi     [n_occ][n_pw_half] device output
 *   E_x    host output (may be NULL)
 * ACE_ERR_NOT_POSDEF if -M is not positive definite.
 */
int ace_build(ace_plan* plan, const void* psi_G, int n_occ, double alpha, const int32_t* pair_row_ptr,
              const int32_t* pair_col, void* xi, double* E_x, void* stream);

/*
 * ace_build without host synchronisation, for CUDA-graph capture and
 * overlapped work: the same work enqueued on `stream` (no Gamma-point check of
 * psi_G: ace_build does it), the status and E_x left in the plan's pinned
 * result slots, read by ace_build_result once the stream (or the graph launch)
 * has completed.
 * Capture: enqueued while `stream` is capturing, the call records its copies
 * and kernels into the graph and allocates nothing; run the same call (same
 * n_occ, same pair list length) once outside capture first, or it fails with
 * ACE_ERR_INVALID_ARG.  A replay reads psi_G, writes xi and uploads the pair
 * list last enqueued on the plan.  ace_apply may be captured the same way.
 * One build per plan at a time: ace_build_result before the next enqueue.
 */
int ace_build_async(ace_plan* plan, const void* psi_G, int n_occ, double alpha, const int32_t* pair_row_ptr,
                    const int32_t* pair_col, void* xi, void* stream);
/* Wait for `stream`, then E_x (may be NULL) of the last enqueued build;
 * ACE_ERR_NOT_POSDEF or ACE_ERR_TIMEOUT as ace_build. */
int ace_build_result(ace_plan* plan, double* E_x, void* stream);

/*
 * The two halves of ace_build, for a build whose pairs are split over several
 * GPUs (the pair terms of Eq. 2-4 are independent; W and E_x are sums over
 * pairs, so the only exchange is one sum over the shards):
 *   ace_build_pairs: phi(r), the Poisson solve of every listed pair and the
 *     exchange accumulation, restricted to this shard's pairs:
 *       W_G    [n_occ][n_pw_half] device output, alpha-scaled V_X Phi over the
 *              listed pairs only (zero where no listed pair touches a row)
 *       E_part host output (may be NULL), -alpha sum (2 - d_ij) e_ij over the
 *              listed pairs
 *     pair_row_ptr/pair_col as in ace_build (all n_occ rows; a shard's rows
 *     may be empty; both NULL = every pair).  Synchronises the stream.
 *   ace_build_finish: with W_G summed over the shards (by the caller, e.g. an
 *     allreduce), M = Phi^T W, -M = L L^T, xi = W L^-T into xi
 *     [n_occ][n_pw_half] device.  ACE_ERR_NOT_POSDEF as ace_build.
 *     Synchronises the stream.
 * When the shards' pair lists partition the full list, summing the shards'
 * W_G and E_part and finishing gives ace_build's xi and E_x up to rounding.
 */
int ace_build_pairs(ace_plan* plan, const void* psi_G, int n_occ, double alpha, const int32_t* pair_row_ptr,
                    const int32_t* pair_col, void* W_G, double* E_part, void* stream);
int ace_build_finish(ace_plan* plan, const void* psi_G, int n_occ, const void* W_G, void* xi, void* stream);

/*
 * Orbital screening of s-MTACE (Section 2.4): the overlaps
 *   S_ij = integral |phi_i(r) phi_j(r)| dr = (Omega / N) sum_r |phi_i(r)| |phi_j(r)|
 * of the real-space orbitals on the plan's grid, and the pairs the paper keeps,
 * S_ij >= rho_cut (i <= j; the diagonal always), as the CSR that ace_build
 * takes.  Single-precision plans form S on the tcgen05 tensor cores (TF32
 * hi/lo split, FP32 slices summed in FP64), double plans on CUDA cores.
 *   psi_G        [n_occ][n_pw_half] device, as ace_build
 *   pair_row_ptr [n_occ + 1] host output
 *   pair_col     host output, room for n_occ (n_occ + 1) / 2 entries
 *   n_pairs      host output (may be NULL): kept pairs
 *   S            [n_occ][n_occ] host output (may be NULL)
 * Synchronises the stream.  Pairs whose S lies within rounding of rho_cut may
 * fall either way.
 */
int ace_overlap_screen(ace_plan* plan, const void* psi_G, int n_occ, double rho_cut, int32_t* pair_row_ptr,
                       int32_t* pair_col, int* n_pairs, double* S, void* stream);

/*
 * SCDM localisation (Section 2.4) with the s'-MTACE pre-selection (Section
 * 2.5): the orthonormal localised orbitals built from selected columns of the
 * density matrix Gamma = Psi Psi^*, for the s-MTACE construction.
 *   1. rho(r) = sum_i psi_i(r)^2 and grad rho = 2 sum_i psi_i grad psi_i on the
 *      plan's grid (grad psi_i exact for the plane-wave expansion);
 *   2. preselect != 0: candidate grid points are those with rho > <rho> and
 *      |grad rho| < <|grad rho|> (averages over all grid points); preselect == 0:
 *      every grid point;
 *   3. column-pivoted (rank-revealing) QR of Psi^* restricted to the candidate
 *      columns: the n_occ pivots C_k, at each step the column of largest
 *      residual norm (ties to the lowest grid index);
 *   4. phi_G = O psi_G with O = (V V^T)^{-1/2} V, V[k][i] = psi_i(r_{C_k}): the
 *      columns Gamma(r, r_{C_k}) orthonormalised symmetrically (Loewdin).
 * Every step after the real-space orbitals runs in double, except that for
 * ACE_MIXED plans the QR's column pass forms q . a (a the single-precision
 * orbital values, exact in float) in float-float arithmetic, about 2^-48 of
 * sum |q_i a_i|, and phi_G = O psi_G is formed in float with compensated sums.
 *   psi_G        [n_occ][n_pw_half] device, orthonormal, as ace_build (n_occ <= 2048)
 *   phi_G        [n_occ][n_pw_half] device output, same precision; must not overlap psi_G
 *   pivots       [n_occ] host output (may be NULL): grid points (i0 n1 + i1) n2 + i2, in pivot order
 *   n_candidates host output (may be NULL): candidate grid points
 *   O            [n_occ][n_occ] host output (may be NULL): the orthogonal rotation, row k for pivot k
 * ACE_ERR_NOT_POSDEF when fewer candidates than orbitals remain, the candidate
 * columns have rank below n_occ, or the orthonormalisation does not converge.
 * Uses the plan's real-space buffers (the next ace_build recomputes them).
 * Synchronises the stream.  Grid points whose rho or |grad rho| lies within
 * rounding of an average, and pivots whose residual ties within rounding, may
 * fall either way.
 */
int ace_scdm(ace_plan* plan, const void* psi_G, int n_occ, int preselect, void* phi_G, int32_t* pivots,
             int* n_candidates, double* O, void* stream);

/*
 * Apply the compressed operator (Eq. 5, an inner MTS step):
 *   Kpsi = -xi (xi^T psi), with the Gamma-point inner product
 *   <a|b> = 2 Re sum_{half} a^* b - a(0) b(0).
 *   xi [n_occ][n_pw_half], psi [T][n_pw_half], Kpsi [T][n_pw_half]: device.
 */
int ace_apply(ace_plan* plan, const void* xi, int n_occ, const void* psi, int T, void* Kpsi, void* stream);

/*
 * Prepare the inner steps of one outer MTS step (Section 2.3): the plan makes
 * a split copy of xi (TF32 hi / lo in the tensor cores' operand tiles, twice
 * xi's size, plan-owned) that later ace_apply calls with the same xi pointer
 * and n_occ read by bulk copies instead of splitting xi themselves (same
 * arithmetic, same results).  The copy is used until the next ace_build /
 * ace_build_async / ace_build_finish / ace_load on the plan or the next
 * ace_apply_prepare; a caller that changes xi's contents by other means must
 * call ace_apply_prepare again.  ACE_FP64 plans and plans with the CUDA-core
 * Gram (ace_opts.kernels = 1) have nothing to prepare and return ACE_OK.
 *   xi [n_occ][n_pw_half] device (read on `stream`).
 */
int ace_apply_prepare(ace_plan* plan, const void* xi, int n_occ, void* stream);

/*
 * The fast energy of an inner MTS step (Section 2.3, Eq. 6-7, with the
 * operator of Eq. 5): E = sum_t <psi_t| K psi_t> = -sum_{t,k} <xi_k|psi_t>^2,
 * from the Gram C = xi^T psi of the apply (no K psi is formed), reduced in
 * FP64 on the device; only E comes back to the host.
 *   xi [n_occ][n_pw_half], psi [T][n_pw_half]: device; E: host output.
 * Synchronises the stream; cannot be captured in a CUDA graph.
 */
int ace_apply_energy(ace_plan* plan, const void* xi, int n_occ, const void* psi, int T, double* E, void* stream);

/*
 * ace_apply for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment variant of the Eq. 5 apply above).
 * Callers in an inner loop that must not stall on cudaMalloc / cudaFree
 * (both synchronise the device), or whose device memory belongs to another
 * allocator, get the operator of ace_apply without a plan and without any
 * allocation: the working memory is a fixed 8 MiB __device__ array inside the
 * library, held on every device that loads the library until the process
 * exits.  For ACE_MIXED it forms xi^T psi on CUDA cores (float products
 * summed in double over short slices) where ace_apply uses the tensor cores,
 * and -xi C with compensated float sums, so it agrees with ace_apply within
 * the parity tolerance (1e-6 of the largest |K psi|), not bit for bit.
 *   xi [n_occ][n_pw_half], psi [T][n_pw_half], Kpsi [T][n_pw_half]: device,
 *   all on the current device, complex128 for precision ACE_FP64, complex64
 *   for ACE_MIXED.
 * Limit: T * n_occ <= 524288, else ACE_ERR_INVALID_ARG and nothing runs.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  All calls share
 * the one array and every call overwrites what it uses, so calls that
 * overlap on the GPU (other streams, other host threads) race: keep them
 * ordered.
 */
int ace_apply_noalloc(const void* xi, int n_occ, const void* psi, int T, int n_pw_half, int precision, void* Kpsi,
                      void* stream);

/*
 * Exact exchange on trial vectors (Eq. 2 with the occupied set psi_occ):
 *   Vx_psi[t] = -alpha sum_j v_{t j} phi_j, projected on the half sphere.
 *   psi_occ [n_occ][n_pw_half], psi [T][n_pw_half], Vx_psi [T][n_pw_half].
 */
int hfx_apply_exact(ace_plan* plan, const void* psi_occ, int n_occ, double alpha, const void* psi, int T,
                    void* Vx_psi, void* stream);

/*
 * Several independent systems (their own plans, sizes and pair lists) built
 * in one call, the batching of independent ACE builds (each system is one
 * ace_build, Section 2.2): the systems' work runs concurrently on streams
 * forked from and joined back into `stream`.  Every plan must be on the same
 * device and distinct.  On return each system carries its E_x and status
 * (ACE_OK or the error ace_build would return); the call returns ACE_OK or the
 * first error.
 */
typedef struct {
    ace_plan* plan;               /* this system's plan */
    const void* psi_G;            /* [n_occ][n_pw_half] device */
    int n_occ;
    double alpha;
    const int32_t* pair_row_ptr;  /* host CSR of kept pairs, or NULL for all */
    const int32_t* pair_col;
    void* xi;                     /* [n_occ][n_pw_half] device output */
    double E_x;                   /* output */
    int status;                   /* output */
} ace_system;

int ace_build_batched(ace_system* systems, int n_sys, void* stream);

/*
 * Checkpoint of the ACE operator between MTS steps (the operator persists
 * across the inner steps, Section 2.3): ace_save writes the vectors xi
 * [n_occ][n_pw_half] (device) with the plan's grid, cell, cutoff, precision,
 * alpha and E_x to a file; ace_load reads them back into xi (device, room for
 * n_occ_max rows) for a plan of the same grid, cell, cutoff and precision,
 * returning n_occ, alpha and E_x (alpha, E_x may be NULL).  Both synchronise
 * the stream.  ACE_ERR_INVALID_ARG on I/O failure or a mismatched file.
 */
int ace_save(const char* path, const ace_plan* plan, const void* xi, int n_occ, double alpha, double E_x,
             void* stream);
int ace_load(const char* path, const ace_plan* plan, void* xi, int* n_occ, double* alpha, double* E_x, void* stream);

/*
 * Intermediates of the last ace_build on this plan (for checking):
 *   W_G [n_occ][n_pw_half] device (alpha-scaled V_X Phi), may be NULL;
 *   M   [n_occ][n_occ] host doubles, may be NULL.  Synchronises the stream.
 */
int ace_last_intermediates(ace_plan* plan, void* W_G, double* M, void* stream);

/*
 * Per-phase device time, from CUDA events recorded while timing is enabled
 * (ace_set_timing), summed over the calls since the last ace_get_stats.  The
 * pair passes run in sub-batches on two streams forked from the call's stream
 * (they overlap); each pass is timed on the stream that runs it, so the three
 * pair phases can add up to more than their wall time.  total_ms is the wall
 * time of the calls on their own stream.  ace_get_stats synchronises with the
 * recorded events and resets the sums.  Counters (transforms, launches) are
 * kept whether timing is on or not.
 */
typedef struct {
    double orbitals_ms;       /* psi_G -> phi(r): scatter and inverse FFT passes */
    double pair_fwd_ms;       /* pair densities and forward FFT passes (Eq. 3) */
    double pair_coulomb_ms;   /* Coulomb passes: forward z, 4 pi / |G|^2, inverse z */
    double pair_inv_ms;       /* inverse FFT passes fused with W accumulation (Eq. 2, 4) */
    double w_to_g_ms;         /* W(r) -> W(G) */
    double gram_ms;           /* Gamma Gram products (M, and xi^T psi in the apply) */
    double factor_ms;         /* Cholesky of -M and the inverse factor */
    double xi_ms;             /* xi = L^-1 W, and -xi C in the apply */
    double energy_ms;         /* E_x reduction */
    double total_ms;          /* wall time of the calls */
    long long pair_transforms;  /* packed pair transforms (two pairs each) */
    long long launches;         /* kernels launched by the library */
    double pair_wall_ms;        /* wall time of the pair passes (all streams) */
} ace_stats;

int ace_set_timing(ace_plan* plan, int enable);
int ace_get_stats(ace_plan* plan, ace_stats* stats);

/*
 * The failure path of the library's bounded device-side waits, exercised
 * without a fault (the paper has no counterpart): one block waits, for at
 * most limit_ms (1 .. 2000), on a barrier that nothing completes, exactly as
 * a bulk copy or a pipeline dependency that never arrives would be waited
 * for.  Returns ACE_ERR_TIMEOUT, as a real time-out does; the plan and the
 * CUDA context stay usable.  Synchronises the stream.
 */
int ace_check_timeout_path(ace_plan* plan, int limit_ms, void* stream);

/* Message of this thread's last error ("" if none); returns its length. */
int ace_last_error(char* buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* ACE_H */
