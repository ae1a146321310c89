// ace_abi.cu -- the C ABI of include/ace.h: plans, workspace, and the order in
// which the kernels run for the ACE build, the ACE apply and the exact
// exchange apply (arXiv:2110.07670 Sections 2.1-2.2, Eq. 2-5).
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ace.h"
#include "internal.h"

using namespace ace;

namespace {

thread_local std::string g_err;
// set while a call enqueues onto a capturing stream: no allocation, no timing
// events, no host synchronisation may happen then
thread_local bool g_capture = false;

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define ACE_CK(expr)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess) return fail(ACE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define ACE_TRY(expr)          \
    do {                       \
        int s_ = (expr);       \
        if (s_ != ACE_OK) return s_; \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool reciprocal(const double a[9], double b[9], double* omega) {
    const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                       a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (!(std::fabs(det) > 0)) return false;
    *omega = std::fabs(det);
    // b_i = 2 pi (a_j x a_k) / det, rows
    const double* r[3] = {a, a + 3, a + 6};
    for (int i = 0; i < 3; ++i) {
        const double* u = r[(i + 1) % 3];
        const double* v = r[(i + 2) % 3];
        b[3 * i + 0] = 2 * M_PI * (u[1] * v[2] - u[2] * v[1]) / det;
        b[3 * i + 1] = 2 * M_PI * (u[2] * v[0] - u[0] * v[2]) / det;
        b[3 * i + 2] = 2 * M_PI * (u[0] * v[1] - u[1] * v[0]) / det;
    }
    return true;
}

int roundup(int x, int m) { return (x + m - 1) / m * m; }

int largest_divisor_at_most(int n, int cap) {
    for (int d = std::min(n, std::max(cap, 1)); d >= 1; --d)
        if (n % d == 0) return d;
    return 1;
}

}  // namespace

struct ace_plan {
    int dev = 0;
    int sms = 152;             // SMs of the plan's device
    int gram_kmax = 0;         // at most this many reals per K slice of the streamed Gram (0: one wave of
                               // blocks; env ACE_GRAM_KMAX)
    float* d_csplit = nullptr; // TF32 hi / lo images of the apply's C (apply_product_scratch floats)
    size_t csplit_cap = 0;
    int prec = ACE_MIXED;
    int n[3] = {0, 0, 0};
    long long N = 0;
    double cell[9], b[9], omega = 0, ecut = 0;
    int n_occ_max = 0;
    std::vector<int32_t> miller;
    int npw = 0;
    int* d_ip = nullptr;
    int* d_in = nullptr;
    AxisPlan ax[3];
    void* d_tw[3] = {nullptr, nullptr, nullptr};
    int* d_freq[3] = {nullptr, nullptr, nullptr};
    bool fused_xy = false;
    bool cube_kernels = true;  // compile-time kernels for supported N^3 boxes
    bool tensor_gram = false;  // Gram products on tcgen05 tensor cores (single precision)
    int lookahead = 1;         // L2 look-ahead of the pair passes, in transforms (env ACE_LOOKAHEAD)
    bool zline = false;        // per-pencil Coulomb pass (zline.cuh) with the kernel table d_kern
    float* d_kern = nullptr;   // 4 pi / |G|^2 / N in the tile passes' spectrum layout (zline only)
    float* d_kern_t = nullptr; // the same for transposed planes (n % 8 == 0 cubes)
    double coul_rc = 0;        // Coulomb cutoff radius (0: 4 pi / |G|^2 with G = 0 dropped)
    int coul_g0 = 0;           // 1: the bare kernel keeps K(0) = 4 pi chi (auxiliary function)
    double coul_k0 = 0;        // that K(0)
    void* d_kern_r = nullptr;  // K(G) / N for the Coulomb stage of the tile passes, R[n0][n1][n2]
    struct Scdm {                 // SCDM workspace, grown on first use
        double* gv = nullptr;     // G components per plane wave [3][npw]
        char* dpsi = nullptr;     // derivative coefficients [n][npw] complex (plan precision)
        double* dens = nullptr;   // rho [N], grad rho [3][N], then the stats partials and means
        int* isel = nullptr;      // block counts, offsets, candidate grid points
        char* A = nullptr;        // candidate columns [n][m] (plan precision)
        double* nu = nullptr;     // residual norms [m], then the QR coefficients [n][m]
        char* part = nullptr;     // argmax partials
        double* mats = nullptr;   // Q, X, T, Y [n][n] each, err, nu0, r [n], c [n]
        int* ipiv = nullptr;      // pivots [n], status
        size_t c_dpsi = 0, c_dens = 0, c_isel = 0, c_A = 0, c_nu = 0, c_part = 0, c_mats = 0, c_ipiv = 0;
    } scdm;
    int variant = 1;           // pair passes: 1 tile, 2 transposed planes, 3 persistent pipeline, 4 hybrid
    bool hybrid = false;       // variant 4: plane-kernel P1 in the tile layout, then the tile P2 / P3
    bool half = false;         // variant 5: P1 / P3 on clusters of two half-plane blocks (halfplane.cuh)
    float tune_ms[6] = {0, 0, 0, 0, 0, 0};  // autotune: tile x1 stream, tile x2, planes x2, pipeline, hybrid x2,
                                          // half planes x2
    float tune_rb_ms[4] = {0, 0, 0, 0};  // autotune of the chosen variant's row block: row order, 2, 4, 8 rows
    int tune_cached = 0;                 // 1: the choice came from the tune cache (ACE_TUNE_CACHE)
    int pair_r0 = 0;                     // first radix of the pair passes' plan on every axis (0: make_axis_plan's)
    float* d_ximg = nullptr;             // split image of a prepared xi (ace_apply_prepare), xi_image_floats
    size_t ximg_cap = 0;
    mutable const void* ximg_src = nullptr;  // the xi it was made from (null: none; builds and loads clear it)
    int ximg_n = 0;
    int r0_cand[4] = {0, 0, 0, 0};       // the first radices the autotuner timed (0: make_axis_plan's)
    float tune_r0_ms[4] = {0, 0, 0, 0};  // the best pair-pass time of each
    int n_r0_cand = 1;
    bool tplane = false;       // pair passes with transposed spectrum planes (plane.cuh; needs zline)
    int pair_tile = 0;         // pairs ordered in pair_tile x pair_tile orbital blocks (0: row by row; env ACE_PAIR_TILE)
    int row_block = 4;         // pairs packed column-shared in blocks of this many rows (pack_pairs_blocked;
                               // < 2: consecutive pairs of the row-ordered list; env ACE_ROW_BLOCK)
    int pair_streams = 2;      // concurrent streams of pair sub-batches
    int pair_sub = 0;          // transforms per sub-batch (0: batch / pair_streams; env ACE_PAIR_SUB)
    bool fused = false;        // the pair passes as one persistent kernel (pipeline.cuh)
    int fused_lag = 2;         // its steps between a transform's passes
    int fused_slots = 8;       // its spectrum ring, transforms
    int fused_flags = 1;       // bit 0: L2 discard of dead planes, bit 1: ticket prefetch (measured slower)
    int* d_pipe = nullptr;     // its counters: [3][ntrans] done, ticket, abort
    size_t pipe_cap = 0;
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_ev;
    cudaEvent_t fork_ev = nullptr;
    PassShape s_xy{}, s_x{}, s_y{}, s_z{};
    int ntiles_last = 1;  // tiles of the pass that accumulates W
    int ntiles_xy = 1;    // ... with the tile or plane passes (2 n for the half-plane pairs)
    int batch = 1;
    size_t esz = 8;  // bytes of one real
    void* d_phi = nullptr;
    void* d_acc = nullptr;
    void* d_spec = nullptr;
    void* d_WG = nullptr;
    double* d_M = nullptr;
    double* d_S = nullptr;     // the overlap screen's S (the last build's M stays in d_M)
    size_t S_cap = 0;
    double* d_L = nullptr;
    double* d_Linv = nullptr;
    double* d_chol = nullptr;  // blocked Cholesky workspace (neg_cholesky_work(n_occ_max) doubles)
    double* d_E = nullptr;
    int* d_status = nullptr;
    int* d_err = nullptr;
    double* d_part = nullptr;
    size_t part_cap = 0;
    Quad* d_quads = nullptr;
    size_t quads_cap = 0;
    double* d_epart = nullptr;
    size_t epart_cap = 0;
    void* d_tphi = nullptr;
    void* d_tacc = nullptr;
    size_t t_cap = 0;
    double* d_C = nullptr;
    size_t C_cap = 0;
    int last_n_occ = 0;
    int pending_n_occ = 0;
    struct Result {
        int status;
        double E;
    };
    Result* h_res = nullptr;  // pinned host slots for the asynchronous build result
    Quad* h_quads = nullptr;  // pinned staging of the quads
    size_t hq_cap = 0;
    cudaEvent_t quads_ev = nullptr;
    // timing: events recorded at phase boundaries; each interval belongs to the
    // phase of the event that opens it (PH_IDLE closes a call)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Mark {
        int phase;
        cudaEvent_t ev;
        int lane;  // 0: the call's stream; k + 1: pair stream k
    };
    std::vector<Mark> marks;
    long long pair_transforms = 0;
    long long launches = 0;
};

namespace {

// PH_PAIRWALL: the wall time of pair passes spread over the pair streams
// (counted in the total only; the passes themselves are timed per stream)
enum Phase { PH_IDLE = -1, PH_ORB = 0, PH_PFWD, PH_PCOUL, PH_PINV, PH_W2G, PH_GRAM, PH_FACTOR, PH_XI, PH_ENERGY,
             PH_PAIRWALL, PH_N };

void mark(ace_plan* P, int phase, cudaStream_t st, int lane = 0) {
    if (!P->timing || g_capture) return;
    cudaEvent_t e;
    if (!P->ev_pool.empty()) {
        e = P->ev_pool.back();
        P->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(e, st);
    P->marks.push_back({phase, e, lane});
}

template <typename T>
int grow(T** p, size_t* cap, size_t need) {
    if (need <= *cap) return ACE_OK;
    if (g_capture)
        return fail(ACE_ERR_INVALID_ARG,
                    "the call needs device memory the plan has not allocated yet; run it once outside stream capture");
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc((void**)p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ACE_ERR_OOM, "device allocation of " + std::to_string(need * sizeof(T)) + " bytes failed");
    }
    *cap = need;
    return ACE_OK;
}

int dalloc(void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ACE_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return ACE_OK;
}

void half_sphere(const double cell[9], const double b[9], double ecut, std::vector<int32_t>& m) {
    int lim[3];
    for (int i = 0; i < 3; ++i) {
        const double len = std::sqrt(cell[3 * i] * cell[3 * i] + cell[3 * i + 1] * cell[3 * i + 1] +
                                     cell[3 * i + 2] * cell[3 * i + 2]);
        lim[i] = (int)std::floor(std::sqrt(ecut) * len / (2 * M_PI)) + 1;
    }
    m.clear();
    for (int h = 0; h <= lim[0]; ++h)
        for (int k = -lim[1]; k <= lim[1]; ++k)
            for (int l = -lim[2]; l <= lim[2]; ++l) {
                if (!(h > 0 || (h == 0 && k > 0) || (h == 0 && k == 0 && l >= 0))) continue;
                double g2 = 0;
                for (int j = 0; j < 3; ++j) {
                    const double g = h * b[j] + k * b[3 + j] + l * b[6 + j];
                    g2 += g * g;
                }
                if (g2 > ecut) continue;
                m.push_back(h);
                m.push_back(k);
                m.push_back(l);
            }
}

template <typename R>
int setup_shapes(ace_plan* P) {
    int smax = 0;
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->dev);
    if (smax <= 0) smax = 227 * 1024;
    const size_t c = sizeof(cx<R>);
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    auto mk_shape = [&](int tz, int ty, int tx, int axes, int threads = 0) {
        PassShape s{};
        s.tz = tz;
        s.ty = ty;
        s.tx = tx;
        s.axes = axes;
        const int e = tz * ty * tx;
        s.threads = threads > 0 ? threads : std::min(512, std::max(128, roundup(e / 24, 32)));
        // bulk copies need 16-byte aligned runs; vectors need 4 consecutive reals
        s.bulk = (c == 16 || (n2 % 2 == 0 && tx % 2 == 0)) ? 1 : 0;
        s.vec = (tx % 4 == 0 && n2 % 4 == 0) ? 1 : 0;
        const int tw = ((axes & 1) ? n2 : 0) + ((axes & 2) ? n1 : 0) + ((axes & 4) ? n0 : 0);
        s.smem = (size_t)e * c + (size_t)tw * c + ((axes & 4) ? (size_t)(n0 + n1 + n2) * 3 * (c / 2) : 0);
        const size_t red = (size_t)(s.threads / 32) * 2 * sizeof(double);
        if (s.smem < red) s.smem = red;
        return s;
    };
    const int target = (int)((64 * 1024) / c);  // elements of a one-axis tile (64 KB)
    const long long plane = (long long)n1 * n2;
    if (P->cube_kernels && c == 8 && n0 == n1 && n1 == n2 && cube_supported(n0)) {
        // compile-time kernels: whole planes and n x ty x tx pencil tiles
        const int n = n0;
        P->fused_xy = true;
        P->s_xy = mk_shape(1, n, n, 3, cube_xy_threads(n));
        P->s_z = mk_shape(n, cube_z_ty(n), cube_z_tx(n), 4, cube_z_threads(n));
        P->s_xy.cube = P->s_z.cube = 1;
        if (P->s_xy.smem > (size_t)smax || P->s_z.smem > (size_t)smax)
            return fail(ACE_ERR_GRID_TOO_SMALL, "plane tile exceeds shared memory");
        P->ntiles_last = P->ntiles_xy = n;
        return ACE_OK;
    }
    P->fused_xy = (size_t)(plane + n1 + n2) * c <= (size_t)std::min(smax, 160 * 1024);
    if (P->fused_xy) P->s_xy = mk_shape(1, n1, n2, 3);
    {
        const int ty = largest_divisor_at_most(n1, std::max(1, target / n2));
        P->s_x = mk_shape(1, ty, n2, 1);
        const int tx = largest_divisor_at_most(n2, std::max(1, std::min(32, target / n1)));
        P->s_y = mk_shape(1, n1, tx, 2);
    }
    {
        const int tx = largest_divisor_at_most(n2, std::max(1, std::min(32, target / n0)));
        const int ty = largest_divisor_at_most(n1, std::max(1, target / (n0 * tx)));
        P->s_z = mk_shape(n0, ty, tx, 4);
    }
    for (const PassShape* s : {&P->s_xy, &P->s_x, &P->s_y, &P->s_z}) {
        if (s == &P->s_xy && !P->fused_xy) continue;
        if (s->smem > (size_t)smax) return fail(ACE_ERR_GRID_TOO_SMALL, "grid axis too long for one thread block tile");
    }
    P->ntiles_last = P->ntiles_xy = P->fused_xy ? n0 : n0 * (n1 / P->s_x.ty);
    return ACE_OK;
}

template <typename R>
PassArgs base_args(const ace_plan* P) {
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n0 = P->n[0];
    a.n1 = P->n[1];
    a.n2 = P->n[2];
    a.pz = P->ax[0];
    a.py = P->ax[1];
    a.px = P->ax[2];
    a.twz = P->d_tw[0];
    a.twy = P->d_tw[1];
    a.twx = P->d_tw[2];
    a.src_tstride = a.dst_tstride = P->N;
    a.src = a.dst = P->d_spec;
    for (int i = 0; i < 9; ++i) a.b[i] = P->b[i];
    a.kscale = 1.0 / (double)P->N;
    a.err = P->d_err;
    a.lookahead = P->lookahead;
    a.kern = P->tplane ? P->d_kern_t : P->d_kern;
    a.kern_inline = P->d_kern_r != nullptr;  // built only for plans without the per-pencil pass
    if (a.kern_inline) a.kern = P->d_kern_r;
    for (int d = 0; d < 3; ++d) a.freq[d] = P->d_freq[d];
    return a;
}

#define ACE_CKL(expr)                                                                                         \
    do {                                                                                                      \
        cudaError_t e_ = (expr);                                                                              \
        ++P->launches;                                                                                        \
        if (e_ != cudaSuccess) return fail(ACE_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// psi (half sphere) -> real-space functions out[a] (quads (a, a, c, c)).
template <typename R>
int run_to_real(ace_plan* P, const cx<R>* psi, const Quad* dq, int ntrans, R* out, cudaStream_t st) {
    PassArgs a = base_args<R>(P);
    a.quads = dq;
    a.accl = out;
    a.scale = 1.0 / std::sqrt(P->omega);
    cx<R>* spec = (cx<R>*)P->d_spec;
    mark(P, PH_ORB, st);
    for (int t0 = 0; t0 < ntrans; t0 += P->batch) {
        const int nb = std::min(P->batch, ntrans - t0);
        a.t0 = t0;
        ACE_CK(cudaMemsetAsync(spec, 0, (size_t)nb * P->N * sizeof(cx<R>), st));
        ACE_CKL(launch_scatter<R>(psi, dq, t0, nb, P->npw, P->d_ip, P->d_in, spec, P->N, st));
        ACE_CKL(launch_pass<R>(a, P->s_z, PRO_LOAD, EPI_STORE, MID_NONE, +1, nb, st));
        if (P->fused_xy) {
            ACE_CKL(launch_pass<R>(a, P->s_xy, PRO_LOAD, EPI_SPLIT, MID_NONE, +1, nb, st));
        } else {
            ACE_CKL(launch_pass<R>(a, P->s_y, PRO_LOAD, EPI_STORE, MID_NONE, +1, nb, st));
            ACE_CKL(launch_pass<R>(a, P->s_x, PRO_LOAD, EPI_SPLIT, MID_NONE, +1, nb, st));
        }
    }
    return ACE_OK;
}

// real-space accumulators acc[a] -> half-sphere coefficients out[a] * s.
template <typename R>
int run_to_recip(ace_plan* P, const R* acc, const Quad* dq, int ntrans, double s, cx<R>* out, cudaStream_t st) {
    PassArgs a = base_args<R>(P);
    a.quads = dq;
    a.fl = acc;
    cx<R>* spec = (cx<R>*)P->d_spec;
    mark(P, PH_W2G, st);
    for (int t0 = 0; t0 < ntrans; t0 += P->batch) {
        const int nb = std::min(P->batch, ntrans - t0);
        a.t0 = t0;
        if (P->fused_xy) {
            ACE_CKL(launch_pass<R>(a, P->s_xy, PRO_PACK2, EPI_STORE, MID_NONE, -1, nb, st));
        } else {
            ACE_CKL(launch_pass<R>(a, P->s_x, PRO_PACK2, EPI_STORE, MID_NONE, -1, nb, st));
            ACE_CKL(launch_pass<R>(a, P->s_y, PRO_LOAD, EPI_STORE, MID_NONE, -1, nb, st));
        }
        ACE_CKL(launch_pass<R>(a, P->s_z, PRO_LOAD, EPI_STORE, MID_NONE, -1, nb, st));
        ACE_CKL(launch_gather<R>(spec, dq, t0, nb, P->npw, P->d_ip, P->d_in, P->N, s, out, st));
    }
    return ACE_OK;
}

// The passes of one batch of nb packed transforms on stream st, with phase
// marks in timing lane `lane`.
template <typename R>
int pair_batch(ace_plan* P, PassArgs& a, int nb, cudaStream_t st, int lane) {
    P->pair_transforms += nb;
    mark(P, PH_PFWD, st, lane);
    if (P->tplane) {
        ACE_CKL(tplane_pair_launch(P->n[0], 0, a, nb, st));
        mark(P, PH_PCOUL, st, lane);
        ACE_CKL(zline_coulomb_launch(P->n[0], a, nb, st));
        mark(P, PH_PINV, st, lane);
        ACE_CKL(tplane_pair_launch(P->n[0], 1, a, nb, st));
    } else if (P->half) {
        ACE_CKL(halfplane_pair_launch(P->n[0], 0, a, nb, st));
        mark(P, PH_PCOUL, st, lane);
        ACE_CKL(zline_coulomb_launch(P->n[0], a, nb, st));
        mark(P, PH_PINV, st, lane);
        ACE_CKL(halfplane_pair_launch(P->n[0], 1, a, nb, st));
    } else if (P->hybrid) {
        ACE_CKL(tplane_pair_launch(P->n[0], 2, a, nb, st));
        mark(P, PH_PCOUL, st, lane);
        ACE_CKL(zline_coulomb_launch(P->n[0], a, nb, st));
        mark(P, PH_PINV, st, lane);
        ACE_CKL(launch_pass<R>(a, P->s_xy, PRO_LOAD, EPI_ACCUM, MID_NONE, +1, nb, st));
    } else if (P->fused_xy) {
        ACE_CKL(launch_pass<R>(a, P->s_xy, PRO_PAIR, EPI_STORE, MID_NONE, -1, nb, st));
        mark(P, PH_PCOUL, st, lane);
        if (P->zline)
            ACE_CKL(zline_coulomb_launch(P->n[0], a, nb, st));
        else
            ACE_CKL(launch_pass<R>(a, P->s_z, PRO_LOAD, EPI_STORE, MID_COULOMB, -1, nb, st));
        mark(P, PH_PINV, st, lane);
        ACE_CKL(launch_pass<R>(a, P->s_xy, PRO_LOAD, EPI_ACCUM, MID_NONE, +1, nb, st));
    } else {
        ACE_CKL(launch_pass<R>(a, P->s_x, PRO_PAIR, EPI_STORE, MID_NONE, -1, nb, st));
        ACE_CKL(launch_pass<R>(a, P->s_y, PRO_LOAD, EPI_STORE, MID_NONE, -1, nb, st));
        mark(P, PH_PCOUL, st, lane);
        ACE_CKL(launch_pass<R>(a, P->s_z, PRO_LOAD, EPI_STORE, MID_COULOMB, -1, nb, st));
        mark(P, PH_PINV, st, lane);
        ACE_CKL(launch_pass<R>(a, P->s_y, PRO_LOAD, EPI_STORE, MID_NONE, +1, nb, st));
        ACE_CKL(launch_pass<R>(a, P->s_x, PRO_LOAD, EPI_ACCUM, MID_NONE, +1, nb, st));
    }
    return ACE_OK;
}

// Pair Poisson solves with fused exchange accumulation (Eq. 2-4).  With
// pair_streams > 1 the transforms go in sub-batches round-robin over that many
// streams forked from st (each with its own spectrum slots), so one
// sub-batch's accumulation pass overlaps the next one's transforms; the
// accumulators take atomic updates, so the streams need no ordering among
// themselves.
template <typename R>
int run_pairs(ace_plan* P, const R* fl, const R* fr, R* accl, R* accr, int symmetric, const Quad* dq, int ntrans,
              double* e_part, cudaStream_t st) {
    PassArgs a = base_args<R>(P);
    a.fl = fl;
    a.fr = fr;
    a.accl = accl;
    a.accr = accr;
    a.symmetric = symmetric;
    a.quads = dq;
    a.e_part = e_part;
    a.r0 = P->pair_r0;  // the spectrum tables were made for this plan
    if (P->fused && ntrans > 0) {
        // one persistent kernel over every transform (pipeline.cuh)
        ACE_TRY(grow(&P->d_pipe, &P->pipe_cap, (size_t)3 * ntrans + 2));
        ACE_CK(cudaMemsetAsync(P->d_pipe, 0, ((size_t)3 * ntrans + 2) * sizeof(int), st));
        PipeArgs pa;
        pa.ntrans = ntrans;
        pa.lag = P->fused_lag;
        pa.slots = std::min(P->batch, P->fused_slots);
        pa.done = P->d_pipe;
        pa.ticket = P->d_pipe + 3 * (size_t)ntrans;
        pa.abort_flag = pa.ticket + 1;
        pa.discard = P->fused_flags & 1;
        pa.prefetch = (P->fused_flags >> 1) & 1;
        a.t0 = 0;
        P->pair_transforms += ntrans;
        mark(P, PH_PAIRWALL, st);
        ACE_CKL(pipeline_pair_launch(P->n[0], a, pa, st));
        return ACE_OK;
    }
    const int S = std::min(P->pair_streams, P->batch);
    if (S <= 1 || ntrans <= 0) {
        for (int t0 = 0; t0 < ntrans; t0 += P->batch) {
            a.t0 = t0;
            ACE_TRY(pair_batch<R>(P, a, std::min(P->batch, ntrans - t0), st, 0));
        }
        return ACE_OK;
    }
    const int b = std::max(1, std::min(P->pair_sub > 0 ? P->pair_sub : P->batch / S, P->batch / S));
    while ((int)P->aux.size() < S) {
        cudaStream_t s2;
        cudaEvent_t e2;
        ACE_CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        P->aux.push_back(s2);
        ACE_CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        P->aux_ev.push_back(e2);
    }
    if (!P->fork_ev) ACE_CK(cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming));
    mark(P, PH_PAIRWALL, st);
    ACE_CK(cudaEventRecord(P->fork_ev, st));
    for (int k = 0; k < S; ++k) ACE_CK(cudaStreamWaitEvent(P->aux[k], P->fork_ev, 0));
    int k = 0;
    for (int t0 = 0; t0 < ntrans; t0 += b, ++k) {
        const int slot = k % S;
        PassArgs a2 = a;
        a2.t0 = t0;
        a2.src = a2.dst = (cx<R>*)P->d_spec + (size_t)slot * b * P->N;
        ACE_TRY(pair_batch<R>(P, a2, std::min(b, ntrans - t0), P->aux[slot], slot + 1));
    }
    for (int j = 0; j < S; ++j) {
        mark(P, PH_IDLE, P->aux[j], j + 1);
        ACE_CK(cudaEventRecord(P->aux_ev[j], P->aux[j]));
        ACE_CK(cudaStreamWaitEvent(st, P->aux_ev[j], 0));
    }
    return ACE_OK;
}

// G[i][j] = <A_i|B_j> (Gamma inner product), double [m][n].
template <typename R>
int gram(ace_plan* P, const cx<R>* A, int m, const cx<R>* B, int n, double* G, cudaStream_t st) {
    const long long K = 2LL * P->npw;
    mark(P, PH_GRAM, st);
    if constexpr (sizeof(R) == 4) {
        if (P->tensor_gram) {
            const long long kc = gram_stream_kchunk(m, n, K, P->sms, P->gram_kmax);
            const int nchunk = (int)((K + kc - 1) / kc);
            // single-precision partials: half the doubles' room is enough
            ACE_TRY(grow(&P->d_part, &P->part_cap, ((size_t)nchunk * m * n + 1) / 2));
            float* part = reinterpret_cast<float*>(P->d_part);
            ACE_CKL(launch_gram_stream((const float*)A, (const float*)B, m, n, K, kc, part, P->d_err, st));
            ACE_CKL(launch_gram_finish_f32(part, nchunk, (const float*)A, (const float*)B, m, n, K, G, n, st));
            return ACE_OK;
        }
    }
    const int tiles = ((m + 63) / 64) * ((n + 63) / 64);
    int nchunk = std::max(1, (2 * 152 + tiles - 1) / tiles);
    nchunk = (int)std::min<long long>(nchunk, std::max<long long>(1, K / 256));
    ACE_TRY(grow(&P->d_part, &P->part_cap, (size_t)nchunk * m * n));
    ACE_CKL(launch_gram_partial<R>((const R*)A, (const R*)B, m, n, K, nchunk, P->d_part, st));
    ACE_CKL(launch_gram_finish<R>(P->d_part, nchunk, (const R*)A, (const R*)B, m, n, K, G, n, st));
    return ACE_OK;
}

std::vector<Quad> orbital_quads(int n) {
    std::vector<Quad> q;
    for (int a = 0; a < n; a += 2) q.push_back(Quad{a, a, a + 1 < n ? a + 1 : -1, a + 1 < n ? a + 1 : -1});
    return q;
}

// Order the pairs (i, j) by blocks of tb x tb orbitals, each block row by row:
// the transforms of one block touch only 2 tb functions and 2 tb accumulators,
// which can stay in L2 between their uses instead of streaming once per pair.
void tile_pairs(std::vector<int>& pa, std::vector<int>& pb, int tb) {
    std::vector<size_t> idx(pa.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
        const int bx = pa[x] / tb, by = pa[y] / tb, cx_ = pb[x] / tb, cy = pb[y] / tb;
        if (bx != by) return bx < by;
        return cx_ < cy;
    });
    std::vector<int> a2(pa.size()), b2(pb.size());
    for (size_t k = 0; k < idx.size(); ++k) {
        a2[k] = pa[idx[k]];
        b2[k] = pb[idx[k]];
    }
    pa.swap(a2);
    pb.swap(b2);
}

void pack_pairs(const std::vector<int>& pa, const std::vector<int>& pb, std::vector<Quad>& q) {
    for (size_t p = 0; p < pa.size(); p += 2) {
        Quad x{pa[p], pb[p], -1, -1};
        if (p + 1 < pa.size()) {
            x.c = pa[p + 1];
            x.d = pb[p + 1];
        }
        q.push_back(x);
    }
}

// Pack the pairs (i, j), i <= j, two per transform in blocks of rb rows.
// Within a block the columns go in ascending order, and the block's rows that
// list column j are paired up, (i1, j) with (i2, j), as the quad
// (j, i1, j, i2): the column orbital is shared by both pairs, so a transform
// reads one fresh function and makes one merged update of the fresh
// accumulator W_j, while the functions and accumulators of the block's rb rows
// are touched by every transform of the block and stay in L2 as the columns
// stream through.  Pairs left unpaired in their column are packed two at a
// time, in row order, after their block.  Every listed pair appears exactly
// once, so the sums of Eq. 2 and 4 are unchanged; only their order differs.
void pack_pairs_blocked(int n, const std::vector<int>& pa, const std::vector<int>& pb, int rb, std::vector<Quad>& q) {
    if (rb < 2) {
        pack_pairs(pa, pb, q);
        return;
    }
    std::vector<std::vector<int>> rows(n);  // columns listed in each row
    for (size_t p = 0; p < pa.size(); ++p) rows[pa[p]].push_back(pb[p]);
    std::vector<std::pair<int, int>> cr;  // (column, row) of one block
    std::vector<int> la, lb;              // unpaired pairs of one block
    for (int r0 = 0; r0 < n; r0 += rb) {
        const int r1 = std::min(n, r0 + rb);
        cr.clear();
        la.clear();
        lb.clear();
        for (int i = r0; i < r1; ++i)
            for (int j : rows[i]) cr.push_back({j, i});
        std::sort(cr.begin(), cr.end());
        for (size_t s = 0; s < cr.size();) {
            size_t e = s;
            while (e < cr.size() && cr[e].first == cr[s].first) ++e;
            const int j = cr[s].first;
            size_t k = s;
            for (; k + 1 < e; k += 2) q.push_back(Quad{j, cr[k].second, j, cr[k + 1].second});
            if (k < e) {
                la.push_back(cr[k].second);
                lb.push_back(j);
            }
            s = e;
        }
        std::vector<size_t> idx(la.size());
        for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return la[x] < la[y]; });
        for (size_t k = 0; k < idx.size(); k += 2) {
            Quad x{la[idx[k]], lb[idx[k]], -1, -1};
            if (k + 1 < idx.size()) {
                x.c = la[idx[k + 1]];
                x.d = lb[idx[k + 1]];
            }
            q.push_back(x);
        }
    }
}

// A bounded device-side wait that gave up leaves a flag; report and clear it.
int check_device_error(ace_plan* P, cudaStream_t st) {
    int err = 0;
    ACE_CK(cudaMemcpyAsync(&err, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    if (err) {
        ACE_CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), st));
        return fail(ACE_ERR_TIMEOUT, "a bounded wait for a bulk copy timed out on the device");
    }
    return ACE_OK;
}

template <typename R>
int check_gamma(ace_plan* P, const void* psi, int n, cudaStream_t st) {
    std::vector<cx<R>> c0(n);
    ACE_CK(cudaMemcpy2DAsync(c0.data(), sizeof(cx<R>), psi, (size_t)P->npw * sizeof(cx<R>), sizeof(cx<R>), n,
                             cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i)
        if (std::fabs((double)c0[i].im) > 1e-6)
            return fail(ACE_ERR_INVALID_ARG, "Im c(G=0) of vector " + std::to_string(i) + " is not zero");
    return ACE_OK;
}

// The quads go through the plan's pinned staging buffer (a captured copy
// reads it when the graph runs).  Outside capture, the previous upload from it
// is waited for before it is rewritten.
// The quads of a call that is never captured (exact exchange, overlap screen,
// SCDM): copied from pageable memory (the copy has taken the data when it
// returns), leaving the pinned staging buffer, which a captured build's
// replays read, to the builds.
int upload_quads_eager(ace_plan* P, const std::vector<Quad>& q, cudaStream_t st) {
    if (g_capture) return fail(ACE_ERR_INVALID_ARG, "this call cannot be captured");
    ACE_TRY(grow(&P->d_quads, &P->quads_cap, q.size()));
    ACE_CK(cudaMemcpyAsync(P->d_quads, q.data(), q.size() * sizeof(Quad), cudaMemcpyHostToDevice, st));
    return ACE_OK;
}

int upload_quads(ace_plan* P, const std::vector<Quad>& q, cudaStream_t st) {
    ACE_TRY(grow(&P->d_quads, &P->quads_cap, q.size()));
    if (!P->quads_ev) ACE_CK(cudaEventCreateWithFlags(&P->quads_ev, cudaEventDisableTiming));
    if (!g_capture) ACE_CK(cudaEventSynchronize(P->quads_ev));
    if (q.size() > P->hq_cap) {
        if (g_capture)
            return fail(ACE_ERR_INVALID_ARG, "pair list longer than any enqueued on this plan outside stream capture");
        if (P->h_quads) cudaFreeHost(P->h_quads);
        P->h_quads = nullptr;
        P->hq_cap = 0;
        if (cudaMallocHost((void**)&P->h_quads, q.size() * sizeof(Quad)) != cudaSuccess) {
            cudaGetLastError();
            return fail(ACE_ERR_OOM, "pinned host allocation failed");
        }
        P->hq_cap = q.size();
    }
    std::memcpy(P->h_quads, q.data(), q.size() * sizeof(Quad));
    ACE_CK(cudaMemcpyAsync(P->d_quads, P->h_quads, q.size() * sizeof(Quad), cudaMemcpyHostToDevice, st));
    if (!g_capture) ACE_CK(cudaEventRecord(P->quads_ev, st));
    return ACE_OK;
}

// Enqueue the pair part of an ACE build on stream st (inputs already
// validated for the Gamma point): phi(r), every listed pair's Poisson solve
// with the exchange accumulation (Eq. 2-4), W -> W_G (into WG) and E_x over
// the listed pairs (into the plan's pinned host slot).
template <typename R>
int pairs_enqueue(ace_plan* P, const void* psi_G, int n_occ, double alpha, const int32_t* rp, const int32_t* col,
                  void* WG_out, cudaStream_t st) {
    std::vector<int> pa, pb;
    if (rp) {
        if (rp[0] != 0) return fail(ACE_ERR_INVALID_ARG, "pair_row_ptr[0] must be 0");
        for (int i = 0; i < n_occ; ++i) {
            if (rp[i + 1] < rp[i]) return fail(ACE_ERR_INVALID_ARG, "pair_row_ptr not monotone");
            for (int t = rp[i]; t < rp[i + 1]; ++t) {
                if (col[t] < i || col[t] >= n_occ) return fail(ACE_ERR_INVALID_ARG, "pair column out of range");
                pa.push_back(i);
                pb.push_back(col[t]);
            }
        }
    } else {
        for (int i = 0; i < n_occ; ++i)
            for (int j = i; j < n_occ; ++j) {
                pa.push_back(i);
                pb.push_back(j);
            }
    }
    std::vector<Quad> oq = orbital_quads(n_occ), q = oq;
    const int n_orb_t = (int)oq.size();
    if (P->pair_tile > 0) {
        tile_pairs(pa, pb, P->pair_tile);
        pack_pairs(pa, pb, q);
    } else {
        pack_pairs_blocked(n_occ, pa, pb, P->row_block, q);
    }
    const int n_pair_t = (int)q.size() - n_orb_t;
    ACE_TRY(upload_quads(P, q, st));
    const Quad* d_oq = P->d_quads;
    const Quad* d_pq = P->d_quads + n_orb_t;

    const cx<R>* psi = (const cx<R>*)psi_G;
    R* phi = (R*)P->d_phi;
    R* acc = (R*)P->d_acc;
    ACE_TRY(run_to_real<R>(P, psi, d_oq, n_orb_t, phi, st));
    ACE_CK(cudaMemsetAsync(acc, 0, (size_t)n_occ * P->N * sizeof(R), st));
    ACE_TRY(grow(&P->d_epart, &P->epart_cap, (size_t)std::max(n_pair_t, 1) * P->ntiles_last * 2));
    ACE_TRY(run_pairs<R>(P, phi, phi, acc, acc, 1, d_pq, n_pair_t, P->d_epart, st));
    mark(P, PH_ENERGY, st);
    ACE_CKL(launch_energy_reduce(P->d_epart, d_pq, n_pair_t, P->ntiles_last, -alpha * P->omega / (double)P->N,
                                 P->d_E, st));
    cx<R>* WG = (cx<R>*)WG_out;
    ACE_TRY(run_to_recip<R>(P, acc, d_oq, n_orb_t, -alpha * std::sqrt(P->omega) / (double)P->N, WG, st));
    ACE_CK(cudaMemcpyAsync(&P->h_res->E, P->d_E, sizeof(double), cudaMemcpyDeviceToHost, st));
    return ACE_OK;
}

// Enqueue the dense part of an ACE build: M = Phi^T W, -M = L L^T, and
// xi = W L^-T (Section 2.2); the Cholesky status lands in the plan's pinned
// host slot.
template <typename R>
int finish_enqueue(ace_plan* P, const void* psi_G, int n_occ, const void* WG_in, void* xi, cudaStream_t st) {
    P->ximg_src = nullptr;  // a prepared image may be of the xi this build overwrites
    const cx<R>* psi = (const cx<R>*)psi_G;
    const cx<R>* WG = (const cx<R>*)WG_in;
    ACE_TRY(gram<R>(P, psi, n_occ, WG, n_occ, P->d_M, st));
    mark(P, PH_FACTOR, st);
    if (n_occ > 64) {  // over many blocks: one block's FP64 rate would take milliseconds
        int nl = 1;
        ACE_CKL(launch_neg_cholesky_blocked(P->d_M, n_occ, P->d_L, P->d_Linv, P->d_status, P->d_chol, &nl, st));
        P->launches += nl - 1;
    } else {
        ACE_CKL(launch_neg_cholesky_inverse(P->d_M, n_occ, P->d_L, P->d_Linv, P->d_status, st));
    }
    mark(P, PH_XI, st);
    if constexpr (sizeof(R) == 4)  // float-float: double-precision accuracy on the FP32 pipes
        ACE_CKL(launch_gemm_nn_ff(P->d_Linv, n_occ, n_occ, (const float*)WG, 2LL * P->npw, 1.0, (float*)xi, true, st));
    else
        ACE_CKL(launch_gemm_nn<R>(P->d_Linv, n_occ, n_occ, (const R*)WG, 2LL * P->npw, 1.0, (R*)xi, true, st, true));
    mark(P, PH_IDLE, st);
    ACE_CK(cudaMemcpyAsync(&P->h_res->status, P->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    P->pending_n_occ = n_occ;
    return ACE_OK;
}

// Enqueue one ACE build on stream st; the status and E_x land in the plan's
// pinned host slots.
template <typename R>
int build_enqueue(ace_plan* P, const void* psi_G, int n_occ, double alpha, const int32_t* rp, const int32_t* col,
                  void* xi, cudaStream_t st) {
    ACE_TRY(pairs_enqueue<R>(P, psi_G, n_occ, alpha, rp, col, P->d_WG, st));
    return finish_enqueue<R>(P, psi_G, n_occ, P->d_WG, xi, st);
}

// Wait for an enqueued build and report its result.
int build_finish(ace_plan* P, double* E_x, cudaStream_t st) {
    ACE_CK(cudaStreamSynchronize(st));
    ACE_TRY(check_device_error(P, st));
    P->last_n_occ = P->pending_n_occ;
    if (E_x) *E_x = P->h_res->E;
    if (P->h_res->status) return fail(ACE_ERR_NOT_POSDEF, "-M is not positive definite (dependent or zero orbitals)");
    return ACE_OK;
}

template <typename R>
int pairs_impl(ace_plan* P, const void* psi_G, int n_occ, double alpha, const int32_t* rp, const int32_t* col,
               void* WG, double* E_part, cudaStream_t st) {
    ACE_TRY(check_gamma<R>(P, psi_G, n_occ, st));
    ACE_TRY(pairs_enqueue<R>(P, psi_G, n_occ, alpha, rp, col, WG, st));
    ACE_CK(cudaStreamSynchronize(st));
    ACE_TRY(check_device_error(P, st));
    if (E_part) *E_part = P->h_res->E;
    return ACE_OK;
}

template <typename R>
int finish_impl(ace_plan* P, const void* psi_G, int n_occ, const void* WG, void* xi, cudaStream_t st) {
    ACE_TRY(check_gamma<R>(P, psi_G, n_occ, st));
    ACE_TRY(finish_enqueue<R>(P, psi_G, n_occ, WG, xi, st));
    return build_finish(P, nullptr, st);
}

template <typename R>
int build_impl(ace_plan* P, const void* psi_G, int n_occ, double alpha, const int32_t* rp, const int32_t* col,
               void* xi, double* E_x, cudaStream_t st) {
    ACE_TRY(check_gamma<R>(P, psi_G, n_occ, st));
    ACE_TRY(build_enqueue<R>(P, psi_G, n_occ, alpha, rp, col, xi, st));
    return build_finish(P, E_x, st);
}

template <typename R>
int hfx_impl(ace_plan* P, const void* psi_occ, int n_occ, double alpha, const void* psi, int T, void* out,
             cudaStream_t st) {
    ACE_TRY(check_gamma<R>(P, psi_occ, n_occ, st));
    ACE_TRY(check_gamma<R>(P, psi, T, st));
    std::vector<Quad> oq = orbital_quads(n_occ), tq = orbital_quads(T), q = oq;
    q.insert(q.end(), tq.begin(), tq.end());
    std::vector<int> pa, pb;
    for (int t = 0; t < T; ++t)
        for (int j = 0; j < n_occ; ++j) {
            pa.push_back(t);
            pb.push_back(j);
        }
    pack_pairs(pa, pb, q);
    const int no = (int)oq.size(), nt = (int)tq.size(), np = (int)q.size() - no - nt;
    ACE_TRY(upload_quads_eager(P, q, st));
    size_t tcap_elems = P->t_cap;
    void* tphi = P->d_tphi;
    if ((size_t)T * P->N > tcap_elems) {
        if (P->d_tphi) cudaFree(P->d_tphi);
        if (P->d_tacc) cudaFree(P->d_tacc);
        P->d_tphi = P->d_tacc = nullptr;
        P->t_cap = 0;
        ACE_TRY(dalloc(&P->d_tphi, (size_t)T * P->N * sizeof(R)));
        ACE_TRY(dalloc(&P->d_tacc, (size_t)T * P->N * sizeof(R)));
        P->t_cap = (size_t)T * P->N;
        tphi = P->d_tphi;
    }
    R* phi = (R*)P->d_phi;
    ACE_TRY(run_to_real<R>(P, (const cx<R>*)psi_occ, P->d_quads, no, phi, st));
    ACE_TRY(run_to_real<R>(P, (const cx<R>*)psi, P->d_quads + no, nt, (R*)tphi, st));
    ACE_CK(cudaMemsetAsync(P->d_tacc, 0, (size_t)T * P->N * sizeof(R), st));
    ACE_TRY(run_pairs<R>(P, (const R*)tphi, phi, (R*)P->d_tacc, nullptr, 0, P->d_quads + no + nt, np, nullptr, st));
    ACE_TRY(run_to_recip<R>(P, (const R*)P->d_tacc, P->d_quads + no, nt, -alpha * std::sqrt(P->omega) / (double)P->N,
                            (cx<R>*)out, st));
    mark(P, PH_IDLE, st);
    ACE_CK(cudaGetLastError());
    return ACE_OK;
}

// s-MTACE screening (Section 2.4): S_ij = integral |phi_i phi_j| dr on the
// grid, (Omega / N) sum_r |phi_i(r)| |phi_j(r)|, a Gram product of |phi| over
// the N grid points (tcgen05 in single precision), then the kept pairs i <= j
// with S_ij >= rho_cut (the diagonal always) as a CSR.
template <typename R>
int overlap_impl(ace_plan* P, const void* psi_G, int n, double rho_cut, int32_t* rp, int32_t* col, int* n_pairs,
                 double* S_out, cudaStream_t st) {
    ACE_TRY(check_gamma<R>(P, psi_G, n, st));
    std::vector<Quad> oq = orbital_quads(n);
    ACE_TRY(upload_quads_eager(P, oq, st));
    ACE_TRY(grow(&P->d_S, &P->S_cap, (size_t)n * n));
    R* phi = (R*)P->d_phi;
    ACE_TRY(run_to_real<R>(P, (const cx<R>*)psi_G, P->d_quads, (int)oq.size(), phi, st));
    const long long K = P->N;
    const double scale = P->omega / (double)P->N;
    mark(P, PH_GRAM, st);
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        if (P->tensor_gram && K % 2 == 0) {
            // the streamed tcgen05 Gram of |phi| (about one block per SM, K
            // slices summed in FP64 by the finish)
            const long long kc = gram_stream_kchunk(n, n, K, P->sms, P->gram_kmax);
            const int nchunk = (int)((K + kc - 1) / kc);
            ACE_TRY(grow(&P->d_part, &P->part_cap, ((size_t)nchunk * n * n + 1) / 2));
            float* part = reinterpret_cast<float*>(P->d_part);
            ACE_CKL(launch_gram_stream((const float*)phi, (const float*)phi, n, n, K, kc, part, P->d_err, st, true));
            ACE_CKL(launch_overlap_finish<float>(part, nchunk, n, scale, P->d_S, st));
            done = true;
        }
    }
    if (!done) {
        const long long tiles = (long long)((n + 63) / 64) * ((n + 63) / 64);
        int nchunk = (int)std::max<long long>(1, (2 * 152 + tiles - 1) / tiles);
        nchunk = (int)std::min<long long>(nchunk, std::max<long long>(1, K / 256));
        ACE_TRY(grow(&P->d_part, &P->part_cap, (size_t)nchunk * n * n));
        ACE_CKL(launch_overlap_partial<R>(phi, n, K, nchunk, P->d_part, st));
        ACE_CKL(launch_overlap_finish<double>(P->d_part, nchunk, n, scale, P->d_S, st));
    }
    mark(P, PH_IDLE, st);
    std::vector<double> S((size_t)n * n);
    ACE_CK(cudaMemcpyAsync(S.data(), P->d_S, S.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    ACE_TRY(check_device_error(P, st));
    int q = 0;
    rp[0] = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = i; j < n; ++j)
            if (i == j || S[(size_t)i * n + j] >= rho_cut) col[q++] = j;
        rp[i + 1] = q;
    }
    if (n_pairs) *n_pairs = q;
    if (S_out) std::memcpy(S_out, S.data(), S.size() * sizeof(double));
    return ACE_OK;
}

// SCDM localisation (Section 2.4) with the s'-MTACE pre-selection (Section
// 2.5): real-space orbitals, rho and grad rho, the candidate grid points,
// column-pivoted QR of Psi^* on them, and phi_G = O psi_G with O the polar
// factor of V[k][i] = psi_i(r_{C_k}) (scdm.cu).  Blocking: the pivot count
// and the Newton-Schulz convergence are read on the host.
template <typename R>
int scdm_impl(ace_plan* P, const void* psi_G, int n, int preselect, void* phi_G, int32_t* pivots, int* n_cand,
              double* O, cudaStream_t st) {
    ACE_TRY(check_gamma<R>(P, psi_G, n, st));
    auto& W = P->scdm;
    const long long N = P->N;
    const int npw = P->npw;
    std::vector<Quad> oq = orbital_quads(n);
    ACE_TRY(upload_quads_eager(P, oq, st));
    R* phi = (R*)P->d_phi;
    ACE_TRY(run_to_real<R>(P, (const cx<R>*)psi_G, P->d_quads, (int)oq.size(), phi, st));
    long long m = N;
    const int* sel = nullptr;
    if (preselect) {
        if (!W.gv) {
            std::vector<double> gv((size_t)3 * npw);
            for (int p = 0; p < npw; ++p)
                for (int c = 0; c < 3; ++c) {
                    double g = 0;
                    for (int ax = 0; ax < 3; ++ax) g += P->miller[3 * p + ax] * P->b[3 * ax + c];
                    gv[(size_t)c * npw + p] = g;
                }
            ACE_TRY(dalloc((void**)&W.gv, gv.size() * sizeof(double)));
            ACE_CK(cudaMemcpy(W.gv, gv.data(), gv.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
        const int ns = scdm_stats_blocks(N), nsel = scdm_select_blocks(N);
        ACE_TRY(grow(&W.dpsi, &W.c_dpsi, (size_t)n * npw * sizeof(cx<R>)));
        ACE_TRY(grow(&W.dens, &W.c_dens, (size_t)4 * N + 2 * ns + 2));
        ACE_TRY(grow(&W.isel, &W.c_isel, (size_t)2 * nsel + 1 + N));
        double *rho = W.dens, *grad = W.dens + N, *part = W.dens + 4 * N, *means = part + 2 * ns;
        int *counts = W.isel, *offsets = W.isel + nsel, *cand = W.isel + 2 * nsel + 1;
        R* dphi = (R*)P->d_acc;
        cx<R>* dpsi = (cx<R>*)W.dpsi;
        // grad rho = 2 sum_i psi_i grad psi_i, one Cartesian component at a time
        for (int d = 0; d < 3; ++d) {
            ACE_CKL(launch_deriv_coeffs<R>((const cx<R>*)psi_G, n, npw, W.gv + (size_t)d * npw, dpsi, st));
            ACE_TRY(run_to_real<R>(P, dpsi, P->d_quads, (int)oq.size(), dphi, st));
            ACE_CKL(launch_orbital_sum<R>(phi, dphi, n, N, grad + d * N, st));
        }
        ACE_CKL(launch_orbital_sum<R>(phi, nullptr, n, N, rho, st));
        ACE_CKL(launch_scdm_stats(rho, grad, N, part, means, st));
        ACE_CKL(launch_scdm_select(rho, grad, N, means, counts, offsets, cand, st));
        int count = 0;
        ACE_CK(cudaMemcpyAsync(&count, offsets + nsel, sizeof(int), cudaMemcpyDeviceToHost, st));
        ACE_CK(cudaStreamSynchronize(st));
        if (count < n)
            return fail(ACE_ERR_NOT_POSDEF, "pre-selection kept " + std::to_string(count) + " grid points for " +
                                                std::to_string(n) + " orbitals");
        m = count;
        sel = cand;
    }
    // column-pivoted QR of the candidate columns: n steps, each a pass over A
    const int qb = scdm_qr_blocks(m, n, (int)sizeof(R));
    ACE_TRY(grow(&W.A, &W.c_A, (size_t)n * m * sizeof(R)));
    ACE_TRY(grow(&W.nu, &W.c_nu, (size_t)m + (size_t)n * m));
    ACE_TRY(grow(&W.part, &W.c_part, (size_t)qb * scdm_argmax_bytes()));
    ACE_TRY(grow(&W.mats, &W.c_mats, (size_t)4 * n * n + 3 * n + 3));
    ACE_TRY(grow(&W.ipiv, &W.c_ipiv, (size_t)2 * n + 1));
    R* A = (R*)W.A;
    double *Q = W.mats, *X = Q + (size_t)n * n, *T = X + (size_t)n * n, *Y = T + (size_t)n * n, *err = Y + (size_t)n * n;
    int *piv = W.ipiv, *status = W.ipiv + n;  // piv: columns of A; grid points after them
    double *rdiag = err + 2 + 2 * n, *fro = rdiag + n;  // after err, nu0, r, c; fro right after rdiag
    const QrWork qw{W.part, W.nu, W.nu + m, Q, err + 2, err + 2 + n, err + 1, rdiag, piv, status};
    ACE_CK(cudaMemsetAsync(status, 0, sizeof(int), st));
    ACE_CKL(launch_gather_columns<R>(phi, n, N, sel, m, A, st));
    ACE_CKL(launch_qr_init<R>(A, n, m, W.nu, W.part, st));
    for (int k = 0; k < n; ++k) ACE_CKL(launch_qr_step<R>(A, n, m, k, qw, st));
    int h_status = 0;
    ACE_CK(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    if (h_status) return fail(ACE_ERR_NOT_POSDEF, "the candidate columns of Psi^* have rank below n_occ");
    // the polar factor of V by scaled Newton-Schulz steps (Chen & Chow): X0 =
    // V / |V|_F has its singular values in (0, 1]; l estimates the smallest,
    // from above, by min_k R[k][k] / |V|_F (an over-estimate only makes a
    // step less aggressive), and follows its image under each step.  Until
    // X X^T = I to 1e-10; the step after that leaves rounding only.
    ACE_CKL(launch_polar_start<R>(A, n, m, piv, X, fro, st));
    std::vector<double> hd((size_t)n + 1);
    ACE_CK(cudaMemcpyAsync(hd.data(), rdiag, ((size_t)n + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    double l = *std::min_element(hd.begin(), hd.begin() + n) / hd[n];
    if (!(l > 0) || l > 1) l = 1;
    bool converged = false;
    for (int it = 0; it < 100 && !converged; ++it) {
        const double alpha = std::sqrt(3.0 / (1.0 + l + l * l));
        ACE_CKL(launch_newton_schulz_step(X, T, Y, n, alpha, err, st));
        l = std::min(1.0, 0.5 * alpha * l * (3.0 - alpha * alpha * l * l));
        double h_err = 0;
        ACE_CK(cudaMemcpyAsync(&h_err, err, sizeof(double), cudaMemcpyDeviceToHost, st));
        ACE_CK(cudaStreamSynchronize(st));
        converged = h_err < 1e-10;
    }
    if (!converged) return fail(ACE_ERR_NOT_POSDEF, "the orthonormalisation of the selected columns did not converge");
    // phi_G = O psi_G: double arithmetic for double plans; single precision
    // with compensated slice sums otherwise (as the ACE apply)
    ACE_CKL(launch_gemm_nn<R>(X, n, n, (const R*)psi_G, 2LL * npw, 1.0, (R*)phi_G, sizeof(R) == 8, st));
    if (pivots) {
        int* grid_pts = W.ipiv + n + 1;
        ACE_CKL(launch_map_pivots(piv, sel, n, grid_pts, st));
        ACE_CK(cudaMemcpyAsync(pivots, grid_pts, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    if (O) ACE_CK(cudaMemcpyAsync(O, X, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    ACE_TRY(check_device_error(P, st));
    if (n_cand) *n_cand = (int)m;
    return ACE_OK;
}

template <typename R>
int apply_impl(ace_plan* P, const void* xi, int n_occ, const void* psi, int T, void* out, cudaStream_t st) {
    ACE_TRY(grow(&P->d_C, &P->C_cap, (size_t)T * n_occ));
    ACE_TRY(gram<R>(P, (const cx<R>*)psi, T, (const cx<R>*)xi, n_occ, P->d_C, st));  // C[t][k] = <psi_t|xi_k>
    mark(P, PH_XI, st);
    if constexpr (sizeof(R) == 4) {
        if (P->tensor_gram) {  // -xi C on the tensor cores
            ACE_TRY(grow(&P->d_csplit, &P->csplit_cap, apply_product_scratch(T, n_occ)));
            // xi's split image, when ace_apply_prepare made one of this xi
            const float* ximg = P->ximg_src == xi && P->ximg_n == n_occ ? P->d_ximg : nullptr;
            ACE_CKL(launch_apply_product(P->d_C, T, n_occ, (const float*)xi, 2LL * P->npw, P->d_csplit, (float*)out,
                                         P->sms, P->d_err, st, ximg));
            mark(P, PH_IDLE, st);
            return ACE_OK;
        }
    }
    ACE_CKL(launch_gemm_nn<R>(P->d_C, T, n_occ, (const R*)xi, 2LL * P->npw, -1.0, (R*)out, false, st));
    mark(P, PH_IDLE, st);
    return ACE_OK;
}

// sum_t <psi_t|K psi_t> = -sum_{t,k} C_tk^2 with C = xi^T psi (the fast
// energy of an inner MTS step): the apply's Gram, reduced on the device.
template <typename R>
int apply_energy_impl(ace_plan* P, const void* xi, int n_occ, const void* psi, int T, double* E, cudaStream_t st) {
    ACE_TRY(grow(&P->d_C, &P->C_cap, (size_t)T * n_occ));
    ACE_TRY(gram<R>(P, (const cx<R>*)psi, T, (const cx<R>*)xi, n_occ, P->d_C, st));
    mark(P, PH_ENERGY, st);
    ACE_CKL(launch_sumsq(P->d_C, (long long)T * n_occ, -1.0, P->d_E, st));
    mark(P, PH_IDLE, st);
    ACE_CK(cudaMemcpyAsync(&P->h_res->E, P->d_E, sizeof(double), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    ACE_TRY(check_device_error(P, st));
    *E = P->h_res->E;
    return ACE_OK;
}

void free_plan(ace_plan* P) {
    if (P->h_res) cudaFreeHost(P->h_res);
    if (P->quads_ev) cudaEventSynchronize(P->quads_ev);
    if (P->h_quads) cudaFreeHost(P->h_quads);
    if (P->quads_ev) cudaEventDestroy(P->quads_ev);
    for (auto& m : P->marks) cudaEventDestroy(m.ev);
    for (auto e : P->ev_pool) cudaEventDestroy(e);
    for (auto s2 : P->aux) cudaStreamDestroy(s2);
    for (auto e : P->aux_ev) cudaEventDestroy(e);
    if (P->fork_ev) cudaEventDestroy(P->fork_ev);
    void* ptrs[] = {P->d_ip, P->d_in, P->d_tw[0], P->d_tw[1], P->d_tw[2], P->d_freq[0], P->d_freq[1], P->d_freq[2], P->d_phi, P->d_acc, P->d_spec,
                    P->d_WG, P->d_M, P->d_S, P->d_L, P->d_Linv, P->d_chol, P->d_E, P->d_status, P->d_err, P->d_part, P->d_quads,
                    P->d_epart, P->d_tphi, P->d_tacc, P->d_C, P->d_kern, P->d_kern_t, P->d_kern_r, P->d_pipe, P->d_csplit, P->d_ximg,
                    P->scdm.gv, P->scdm.dpsi, P->scdm.dens, P->scdm.isel, P->scdm.A, P->scdm.nu,
                    P->scdm.part, P->scdm.mats, P->scdm.ipiv};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete P;
}

void set_variant(ace_plan* P, int v, int streams) {
    P->variant = v;
    P->tplane = v == 2 || v == 3;
    P->fused = v == 3;
    P->hybrid = v == 4;
    P->half = v == 5;
    P->ntiles_last = v == 5 ? 2 * P->n[0] : P->ntiles_xy;  // one energy partial per half-plane block
    P->pair_streams = streams;
}

// The pair-pass variant (ace_opts.pair_variant): forced, or, when 0 and more
// than one applies, timed on this plan's own buffers (zeroed functions, the
// first transforms of the full pair list of n_occ_max orbitals, one warm-up
// and two timed runs each) and the fastest kept.
template <typename R>
int pair_tables(ace_plan* P, int r0);

// First radix of the pair passes' plan: r0, or make_axis_plan's for r0 = 0.
int first_radix(const ace_plan* P, int r0) { return r0 ? r0 : (P->ax[0].nstages > 0 ? P->ax[0].radix[0] : 1); }

template <typename R>
int choose_pair_variant(ace_plan* P, const ace_opts* opts) {
    const int req = opts ? opts->pair_variant : 0;
    // the pair passes' radix plans: make_axis_plan's (r0 = 0), then the
    // alternatives with compile-time kernels (single-precision cube plans);
    // ACE_PAIR_RADIX=<first radix> keeps one of them
    int r0s[4] = {0, 0, 0, 0};
    int nr0 = 1;
    if (sizeof(R) == 4 && P->zline && P->cube_kernels) nr0 += pair_radix_alternatives(P->n[0], r0s + 1);
    if (const char* env = std::getenv("ACE_PAIR_RADIX")) {
        const int want = std::atoi(env);
        int hit = -1;
        for (int k = 0; k < nr0; ++k)
            if (first_radix(P, r0s[k]) == want) hit = k;
        if (hit < 0) return fail(ACE_ERR_INVALID_ARG, "ACE_PAIR_RADIX names no pair radix plan of this grid");
        r0s[0] = r0s[hit];
        nr0 = 1;
        ACE_TRY(pair_tables<R>(P, r0s[0]));
    }
    P->n_r0_cand = nr0;
    for (int k = 0; k < 4; ++k) P->r0_cand[k] = k < nr0 ? r0s[k] : 0;
    const int fixed_streams = opts && opts->pair_streams > 0 ? opts->pair_streams : 0;
    const bool t_ok = sizeof(R) == 4 && P->zline && P->d_kern_t != nullptr;
    const bool p_ok = t_ok && pipeline_supported(P->n[0]);
    const bool h_ok = sizeof(R) == 4 && P->zline;  // every compile-time cube
    const bool c_ok = h_ok && halfplane_supported(P->n[0]);
    if (req < 0 || req > 5) return fail(ACE_ERR_INVALID_ARG, "pair_variant must be 0 (automatic), 1, 2, 3, 4 or 5");
    if (req == 5 && !c_ok)
        return fail(ACE_ERR_INVALID_ARG, "pair_variant 5 needs a single-precision 120^3 plan");
    if (req == 2 && !t_ok)
        return fail(ACE_ERR_INVALID_ARG,
                    "pair_variant 2 needs a single-precision n^3 plan with n in {32, 80, 96, 120, 160}");
    if (req == 3 && !p_ok)
        return fail(ACE_ERR_INVALID_ARG, "pair_variant 3 needs a single-precision n^3 plan with n in {32, 80, 96, 160}");
    if (req == 4 && !h_ok)
        return fail(ACE_ERR_INVALID_ARG,
                    "pair_variant 4 needs a single-precision n^3 plan with n in {32, 60, 80, 90, 96, 100, 108, 120, 160}");
    if (req > 0) {
        set_variant(P, req, fixed_streams ? fixed_streams : 2);
        return ACE_OK;
    }
    struct Cand {
        int v, streams, slot;
    };
    std::vector<Cand> cand;
    if (!fixed_streams || fixed_streams == 1) cand.push_back({1, 1, 0});
    if (!fixed_streams || fixed_streams >= 2) cand.push_back({1, fixed_streams ? fixed_streams : 2, 1});
    if (t_ok) cand.push_back({2, fixed_streams ? fixed_streams : 2, 2});
    if (p_ok) cand.push_back({3, 1, 3});
    if (h_ok) cand.push_back({4, fixed_streams ? fixed_streams : 2, 4});
    if (c_ok) cand.push_back({5, fixed_streams ? fixed_streams : 2, 5});
    if (sizeof(R) != 4 || cand.size() == 1) {  // double plans: no timing, the two-stream tile passes
        set_variant(P, 1, fixed_streams ? fixed_streams : 2);
        return ACE_OK;
    }
    // the tune cache: one line per (grid, n_occ_max, precision, device)
    char key[256] = {0};
    const char* cache = std::getenv("ACE_TUNE_CACHE");
    if (cache && *cache && !fixed_streams) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, P->dev) != cudaSuccess) {
            cudaGetLastError();
            prop.name[0] = 0;
        }
        for (char* c = prop.name; *c; ++c)
            if (*c == ' ') *c = '_';
        std::snprintf(key, sizeof key, "%dx%dx%d n%d f%d %s sm%d", P->n[0], P->n[1], P->n[2], P->n_occ_max,
                      (int)sizeof(R) * 8, prop.name, P->sms);
        if (FILE* f = std::fopen(cache, "r")) {
            char line[512];
            int v = 0, st = 0, rb = -1, r0 = 0;
            bool hit = false;
            while (std::fgets(line, sizeof line, f)) {
                const size_t kl = std::strlen(key);
                int v2, s2, rb2, r2 = 0;
                const int got = std::strncmp(line, key, kl) == 0 && line[kl] == ' '
                                    ? std::sscanf(line + kl, " = %d %d %d %d", &v2, &s2, &rb2, &r2)
                                    : 0;
                bool r_ok = false;  // the radix plan (a fourth field; 0 when absent) is one of this plan's
                for (int k = 0; k < nr0; ++k) r_ok = r_ok || r0s[k] == r2;
                if ((got == 3 || got == 4) && v2 >= 1 && v2 <= 5 && s2 >= 1 && s2 <= 8 && rb2 >= 0 && rb2 <= 64 &&
                    (v2 != 2 || t_ok) && (v2 != 3 || p_ok) && (v2 != 4 || h_ok) && (v2 != 5 || c_ok) && r_ok) {
                    v = v2;  // the last matching line wins
                    st = s2;
                    rb = rb2;
                    r0 = r2;
                    hit = true;
                }
            }
            std::fclose(f);
            if (hit) {
                if (r0 != P->pair_r0) ACE_TRY(pair_tables<R>(P, r0));
                set_variant(P, v, st);
                P->row_block = rb;
                P->tune_cached = 1;
                return ACE_OK;
            }
        }
    }
    // timing pairs: the first transforms of every pair i <= j of n_occ_max
    // rows, packed as a build packs them
    const int n = P->n_occ_max;
    std::vector<int> pa, pb;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            pa.push_back(i);
            pb.push_back(j);
        }
    const size_t want = (size_t)std::min(4 * P->batch, std::max(1, n * (n + 1) / 4));
    auto quads_for = [&](int rb) {
        std::vector<Quad> q;
        pack_pairs_blocked(n, pa, pb, rb, q);
        q.resize(std::min(q.size(), want));
        return q;
    };
    cudaStream_t ts = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&] {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ts) cudaStreamDestroy(ts);
    };
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(ACE_ERR_CUDA, "autotune: stream or event creation failed");
    }
    // ms per run of the current variant on quads q (one warm-up, two timed runs)
    auto time_runs = [&](const std::vector<Quad>& q, float* out) -> int {
        const int K = (int)q.size();
        ACE_TRY(upload_quads(P, q, ts));
        ACE_TRY(grow(&P->d_epart, &P->epart_cap, (size_t)K * P->ntiles_last * 2));
        R* phi = (R*)P->d_phi;
        R* acc = (R*)P->d_acc;
        for (int rep = 0; rep < 3; ++rep) {
            if (rep == 1 && cudaEventRecord(e0, ts) != cudaSuccess) return fail(ACE_ERR_CUDA, "autotune: event");
            ACE_TRY(run_pairs<R>(P, phi, phi, acc, acc, 1, P->d_quads, K, P->d_epart, ts));
        }
        float ms = 0;
        if (cudaEventRecord(e1, ts) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return fail(ACE_ERR_CUDA, "autotune: timing failed");
        *out = ms / 2;
        return ACE_OK;
    };
    int rc = ACE_OK;
    float best = 1e30f;
    int best_v = 1, best_s = 2, best_rb = P->row_block, best_r0 = P->pair_r0;
    float var_ms[4][6] = {};  // per radix plan and variant slot
    do {
        if (cudaMemsetAsync(P->d_phi, 0, (size_t)n * P->N * sizeof(R), ts) != cudaSuccess ||
            cudaMemsetAsync(P->d_acc, 0, (size_t)n * P->N * sizeof(R), ts) != cudaSuccess) {
            rc = fail(ACE_ERR_CUDA, "autotune: memset failed");
            break;
        }
        const std::vector<Quad> q = quads_for(P->row_block);
        // every radix plan with every variant
        for (int k = 0; k < nr0 && rc == ACE_OK; ++k) {
            if (r0s[k] != P->pair_r0 && (rc = pair_tables<R>(P, r0s[k])) != ACE_OK) break;
            float best_k = 1e30f;
            for (const Cand& c : cand) {
                set_variant(P, c.v, c.streams);
                float ms = 0;
                if ((rc = time_runs(q, &ms)) != ACE_OK) break;
                var_ms[k][c.slot] = ms;
                best_k = std::min(best_k, ms);
                if (ms < best) {
                    best = ms;
                    best_v = c.v;
                    best_s = c.streams;
                    best_r0 = r0s[k];
                }
            }
            P->tune_r0_ms[k] = best_k;
        }
        if (rc != ACE_OK) break;
        for (int k = 0; k < nr0; ++k)
            if (r0s[k] == best_r0)
                for (int v = 0; v < 6; ++v) P->tune_ms[v] = var_ms[k][v];
        if (best_r0 != P->pair_r0 && (rc = pair_tables<R>(P, best_r0)) != ACE_OK) break;
        // then the pair-tile shape of the chosen kernels: row order, or column-
        // shared transforms in blocks of 2, 4 or 8 rows (pack_pairs_blocked)
        if (!std::getenv("ACE_ROW_BLOCK")) {
            set_variant(P, best_v, best_s);
            const int rbs[4] = {0, 2, 4, 8};
            float best_rb_ms = 1e30f;
            for (int k = 0; k < 4 && rc == ACE_OK; ++k) {
                float ms = 0;
                if ((rc = time_runs(quads_for(rbs[k]), &ms)) != ACE_OK) break;
                P->tune_rb_ms[k] = ms;
                if (ms < best_rb_ms) {
                    best_rb_ms = ms;
                    best_rb = rbs[k];
                }
            }
        }
        if (rc == ACE_OK) rc = check_device_error(P, ts);
    } while (false);
    cleanup();
    set_variant(P, best_v, best_s);
    P->row_block = best_rb;
    P->pair_transforms = 0;
    P->launches = 0;
    if (rc == ACE_OK && key[0]) {
        if (FILE* f = std::fopen(cache, "a")) {
            std::fprintf(f, "%s = %d %d %d %d\n", key, best_v, best_s, best_rb, best_r0);
            std::fclose(f);
        }
    }
    return rc;
}

// K(0) = 4 pi chi of the auxiliary-function treatment of the G = 0 term for
// Gamma-only sampling (Gygi & Baldereschi), F(q) = exp(-a q^2) / q^2:
//   chi = Omega / (2 pi)^3 int F d^3q - [sum_{G != 0} F(G) - a]
// (the bracket's -a: F's regular part F - 1/q^2 at q = 0, the G = 0 member
// of the lattice sum).  With a = (L_min / 12)^2 the real-space images of F are
// below double resolution and chi does not depend on a; the sum runs over
// every reciprocal lattice vector with a G^2 <= 50.
double auxiliary_function_k0(const double cell[9], const double b[9], double omega) {
    double lmin = 1e300;
    for (int i = 0; i < 3; ++i)
        lmin = std::min(lmin, std::sqrt(cell[3 * i] * cell[3 * i] + cell[3 * i + 1] * cell[3 * i + 1] +
                                        cell[3 * i + 2] * cell[3 * i + 2]));
    const double a = (lmin / 12.0) * (lmin / 12.0), g2max = 50.0 / a;
    int lim[3];
    for (int i = 0; i < 3; ++i) {
        const double len = std::sqrt(cell[3 * i] * cell[3 * i] + cell[3 * i + 1] * cell[3 * i + 1] +
                                     cell[3 * i + 2] * cell[3 * i + 2]);
        lim[i] = (int)std::ceil(std::sqrt(g2max) * len / (2 * M_PI)) + 1;
    }
    double lattice = 0;
    for (int h = -lim[0]; h <= lim[0]; ++h)
        for (int k = -lim[1]; k <= lim[1]; ++k)
            for (int l = -lim[2]; l <= lim[2]; ++l) {
                if (h == 0 && k == 0 && l == 0) continue;
                double g2 = 0;
                for (int c = 0; c < 3; ++c) {
                    const double g = h * b[c] + k * b[3 + c] + l * b[6 + c];
                    g2 += g * g;
                }
                lattice += std::exp(-a * g2) / g2;
            }
    const double integral = omega / std::pow(2 * M_PI, 3) * 2.0 * std::pow(M_PI, 1.5) / std::sqrt(a);
    return 4 * M_PI * (integral - (lattice - a));
}

// The pair passes' spectrum tables for the radix plan whose first stage has
// radix r0 on every axis (0: make_axis_plan's plan, the one the orbital and W
// transforms use): the frequency at every position (the tile passes' Coulomb
// stage) and the Coulomb factors K(G) / N (Eq. 3) at every stored position,
// computed in double: the per-pencil pass always reads one; the Coulomb stage
// of the tile passes reads one for the cut-off interaction and in double
// precision (one load is cheaper than a double division there); in single
// precision it forms 4 pi / |G|^2 from G itself.  Device buffers are made on
// the first call and rewritten by later ones (the autotuner times each plan).
template <typename R>
int pair_tables(ace_plan* P, int r0) {
    std::vector<int> frq[3];
    for (int d = 0; d < 3; ++d) {
        AxisPlan ax = P->ax[d];
        if (r0 != 0 && !make_axis_plan_first(P->n[d], r0, ax))
            return fail(ACE_ERR_INVALID_ARG, "pair radix plan: the radix does not split the grid into two codelets");
        frq[d].resize(P->n[d]);
        for (int k = 0; k < P->n[d]; ++k) frq[d][digit_reversed_position(ax, k)] = k;
        if (!P->d_freq[d]) ACE_TRY(dalloc((void**)&P->d_freq[d], P->n[d] * sizeof(int)));
        ACE_CK(cudaMemcpy(P->d_freq[d], frq[d].data(), P->n[d] * sizeof(int), cudaMemcpyHostToDevice));
    }
    P->pair_r0 = r0;
    const bool swz = P->s_xy.cube && cube_swizzle(P->n[2]);
    const bool inline_tab = !P->zline && (P->coul_rc > 0 || P->coul_g0 || sizeof(R) == 8);
    if (!P->zline && !inline_tab) return ACE_OK;
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    const bool with_t = P->zline && tplane_supported(n0);
    const bool swz_i = P->s_z.cube && cube_swizzle(n2);  // x slots of the tile passes' Coulomb stage
    std::vector<float> kern(P->zline ? (size_t)P->N : 0), kern_t(with_t ? (size_t)P->N : 0);
    std::vector<R> kern_r(inline_tab ? (size_t)P->N : 0);
    auto fold = [](int k, int n) { return k < n - n / 2 ? k : k - n; };
    auto g2_at = [&](int z, int y, int xp) {
        const int m[3] = {fold(frq[0][z], n0), fold(frq[1][y], n1), fold(frq[2][xp], n2)};
        double q2 = 0;
        for (int c = 0; c < 3; ++c) {
            const double g = m[0] * P->b[c] + m[1] * P->b[3 + c] + m[2] * P->b[6 + c];
            q2 += g * g;
        }
        return q2;
    };
    // 4 pi / |G|^2 with G = 0 dropped, or the transform of 1/r cut off at
    // R_c: 4 pi (1 - cos(|G| R_c)) / |G|^2, and 2 pi R_c^2 at G = 0
    const double rc = P->coul_rc;
    auto k = [&](double q2) {
        if (rc > 0)
            return (q2 > 0 ? 4 * M_PI * (1 - std::cos(std::sqrt(q2) * rc)) / q2 : 2 * M_PI * rc * rc) / (double)P->N;
        return q2 > 0 ? 4 * M_PI / (q2 * (double)P->N) : P->coul_k0 / (double)P->N;
    };
    for (int z = 0; z < n0; ++z)
        for (int y = 0; y < n1; ++y)
            for (int xs = 0; xs < n2; ++xs) {
                const size_t e = ((size_t)z * n1 + y) * n2 + xs;
                if (P->zline) kern[e] = (float)k(g2_at(z, y, swz ? plane_swizzle(xs, y, n2) : xs));
                if (with_t) kern_t[((size_t)z * n2 + xs) * n1 + y] = (float)k(g2_at(z, y, xs));  // plane [x][y]
                if (inline_tab) kern_r[e] = (R)k(g2_at(z, y, swz_i ? plane_swizzle(xs, y, n2) : xs));
            }
    if (with_t) {
        if (!P->d_kern_t) ACE_TRY(dalloc((void**)&P->d_kern_t, kern_t.size() * sizeof(float)));
        ACE_CK(cudaMemcpy(P->d_kern_t, kern_t.data(), kern_t.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (P->zline) {
        if (!P->d_kern) ACE_TRY(dalloc((void**)&P->d_kern, kern.size() * sizeof(float)));
        ACE_CK(cudaMemcpy(P->d_kern, kern.data(), kern.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (inline_tab) {
        if (!P->d_kern_r) ACE_TRY(dalloc(&P->d_kern_r, kern_r.size() * sizeof(R)));
        ACE_CK(cudaMemcpy(P->d_kern_r, kern_r.data(), kern_r.size() * sizeof(R), cudaMemcpyHostToDevice));
    }
    return ACE_OK;
}

template <typename R>
int create_impl(ace_plan* P, const ace_opts* opts) {
    P->esz = sizeof(R);
    for (int d = 0; d < 3; ++d) {
        if (!make_axis_plan(P->n[d], P->ax[d]))
            return fail(ACE_ERR_GRID_TOO_SMALL, "grid extents must be products of 2, 3 and 5");
        std::vector<cx<R>> tw(P->n[d]);
        for (int j = 0; j < P->n[d]; ++j) {
            tw[j].re = (R)std::cos(2 * M_PI * j / P->n[d]);
            tw[j].im = (R)-std::sin(2 * M_PI * j / P->n[d]);
        }
        ACE_TRY(dalloc(&P->d_tw[d], tw.size() * sizeof(cx<R>)));
        ACE_CK(cudaMemcpy(P->d_tw[d], tw.data(), tw.size() * sizeof(cx<R>), cudaMemcpyHostToDevice));
    }
    // digit-reversed positions of every frequency, per axis (the orbital and
    // W transforms' plan)
    std::vector<int> pos[3];
    for (int d = 0; d < 3; ++d) {
        pos[d].resize(P->n[d]);
        for (int k = 0; k < P->n[d]; ++k) pos[d][k] = digit_reversed_position(P->ax[d], k);
    }
    if (opts && opts->kernels >= 2) P->cube_kernels = false;  // generic runtime-size FFT passes
    P->tensor_gram = !(opts && opts->kernels >= 1) && sizeof(R) == 4;
    if (const char* env = std::getenv("ACE_LOOKAHEAD")) P->lookahead = std::max(0, std::atoi(env));
    if (const char* env = std::getenv("ACE_PAIR_TILE")) P->pair_tile = std::max(0, std::atoi(env));
    if (const char* env = std::getenv("ACE_ROW_BLOCK")) P->row_block = std::max(0, std::atoi(env));
    if (const char* env = std::getenv("ACE_GRAM_KMAX")) P->gram_kmax = std::max(0, std::atoi(env));
    {
        int sm_count = 0;
        if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, P->dev) == cudaSuccess && sm_count > 0)
            P->sms = sm_count;
    }
    if (opts && opts->pair_streams > 0) P->pair_streams = opts->pair_streams;
    if (const char* env = std::getenv("ACE_PAIR_SUB")) P->pair_sub = std::max(0, std::atoi(env));
    ACE_TRY(setup_shapes<R>(P));
    // the compile-time plane kernels of N % 16 == 0 boxes keep x swizzled per row
    const bool swz = P->s_xy.cube && cube_swizzle(P->n[2]);
    if (opts) {
        P->coul_rc = opts->coulomb_rc;
        P->coul_g0 = opts->coulomb_g0;
        if (P->coul_g0) P->coul_k0 = auxiliary_function_k0(P->cell, P->b, P->omega);
    }
    P->zline = P->s_xy.cube && P->s_z.cube && zline_group(P->n[0]) > 0;
    if (const char* env = std::getenv("ACE_ZLINE")) P->zline = P->zline && std::atoi(env) != 0;
    ACE_TRY(pair_tables<R>(P, 0));
    std::vector<int> ip(P->npw), in(P->npw);
    for (int p = 0; p < P->npw; ++p) {
        int m[3], mn[3];
        for (int d = 0; d < 3; ++d) {
            const int v = P->miller[3 * p + d];
            m[d] = pos[d][((v % P->n[d]) + P->n[d]) % P->n[d]];
            mn[d] = pos[d][((-v % P->n[d]) + P->n[d]) % P->n[d]];
        }
        if (swz) {
            m[2] = plane_swizzle(m[2], m[1], P->n[2]);
            mn[2] = plane_swizzle(mn[2], mn[1], P->n[2]);
        }
        ip[p] = (m[0] * P->n[1] + m[1]) * P->n[2] + m[2];
        in[p] = (mn[0] * P->n[1] + mn[1]) * P->n[2] + mn[2];
    }
    ACE_TRY(dalloc((void**)&P->d_ip, P->npw * sizeof(int)));
    ACE_TRY(dalloc((void**)&P->d_in, P->npw * sizeof(int)));
    ACE_CK(cudaMemcpy(P->d_ip, ip.data(), P->npw * sizeof(int), cudaMemcpyHostToDevice));
    ACE_CK(cudaMemcpy(P->d_in, in.data(), P->npw * sizeof(int), cudaMemcpyHostToDevice));
    int ntrans_min = (P->n_occ_max + 1) / 2;
    int batch = opts && opts->pair_batch > 0 ? opts->pair_batch
                                             : (int)std::max<long long>(1, (512LL << 20) / (P->N * (long long)sizeof(cx<R>)));
    batch = std::min(batch, 64);
    (void)ntrans_min;
    P->batch = std::max(1, batch);
    const size_t N = (size_t)P->N;
    ACE_TRY(dalloc(&P->d_phi, (size_t)P->n_occ_max * N * sizeof(R)));
    ACE_TRY(dalloc(&P->d_acc, (size_t)P->n_occ_max * N * sizeof(R)));
    ACE_TRY(dalloc(&P->d_spec, (size_t)P->batch * N * sizeof(cx<R>)));
    ACE_TRY(dalloc(&P->d_WG, (size_t)P->n_occ_max * P->npw * sizeof(cx<R>)));
    const size_t nn = (size_t)P->n_occ_max * P->n_occ_max;
    ACE_TRY(dalloc((void**)&P->d_M, nn * sizeof(double)));
    ACE_TRY(dalloc((void**)&P->d_L, nn * sizeof(double)));
    ACE_TRY(dalloc((void**)&P->d_Linv, nn * sizeof(double)));
    ACE_TRY(dalloc((void**)&P->d_chol, neg_cholesky_work(P->n_occ_max) * sizeof(double)));
    ACE_TRY(dalloc((void**)&P->d_E, (1 + 16384) * sizeof(double)));  // E_x, then the energy reduction's block sums
    ACE_TRY(dalloc((void**)&P->d_status, sizeof(int)));
    ACE_TRY(dalloc((void**)&P->d_err, sizeof(int)));
    if (cudaMallocHost((void**)&P->h_res, sizeof(ace_plan::Result)) != cudaSuccess) {
        cudaGetLastError();
        P->h_res = nullptr;
        return fail(ACE_ERR_OOM, "pinned host allocation failed");
    }
    ACE_CK(cudaMemset(P->d_err, 0, sizeof(int)));
    return choose_pair_variant<R>(P, opts);
}

}  // namespace

extern "C" {

int ace_plan_create(ace_plan** plan, const int grid[3], const double cell[9], double ecut_ry, int n_occ_max,
                    int precision, const ace_opts* opts) {
    if (!plan || !grid || !cell) return fail(ACE_ERR_INVALID_ARG, "null argument");
    *plan = nullptr;
    if (!(ecut_ry > 0) || n_occ_max < 1 || (precision != ACE_FP64 && precision != ACE_MIXED))
        return fail(ACE_ERR_INVALID_ARG, "ecut must be > 0, n_occ_max >= 1, precision ACE_FP64 or ACE_MIXED");
    for (int d = 0; d < 3; ++d)
        if (grid[d] < 1 || grid[d] > 4096) return fail(ACE_ERR_INVALID_ARG, "grid extent out of range");
    if (opts && !(std::isfinite(opts->coulomb_rc) && opts->coulomb_rc >= 0))
        return fail(ACE_ERR_INVALID_ARG, "coulomb_rc must be finite and >= 0");
    if (opts && (opts->coulomb_g0 < 0 || opts->coulomb_g0 > 1 || (opts->coulomb_g0 && opts->coulomb_rc > 0)))
        return fail(ACE_ERR_INVALID_ARG, "coulomb_g0 must be 0 or 1, and 0 with coulomb_rc > 0");
    ace_plan* P = new ace_plan();
    cudaGetDevice(&P->dev);
    P->prec = precision;
    for (int d = 0; d < 3; ++d) P->n[d] = grid[d];
    P->N = (long long)grid[0] * grid[1] * grid[2];
    std::memcpy(P->cell, cell, sizeof(P->cell));
    P->ecut = ecut_ry;
    P->n_occ_max = n_occ_max;
    if (!reciprocal(cell, P->b, &P->omega)) {
        delete P;
        return fail(ACE_ERR_INVALID_ARG, "singular cell");
    }
    half_sphere(P->cell, P->b, ecut_ry, P->miller);
    P->npw = (int)(P->miller.size() / 3);
    for (int p = 0; p < P->npw; ++p)
        for (int d = 0; d < 3; ++d)
            if (2 * std::abs(P->miller[3 * p + d]) + 1 > P->n[d]) {
                delete P;
                return fail(ACE_ERR_GRID_TOO_SMALL, "grid too small for the cutoff sphere");
            }
    int st = precision == ACE_FP64 ? create_impl<double>(P, opts) : create_impl<float>(P, opts);
    if (st != ACE_OK) {
        free_plan(P);
        return st;
    }
    *plan = P;
    return ACE_OK;
}

void ace_plan_destroy(ace_plan* plan) {
    if (!plan) return;
    DeviceGuard g(plan->dev);
    free_plan(plan);
}

int ace_gvec(const ace_plan* plan, int* n_pw_half, int32_t* miller) {
    if (!plan || !n_pw_half) return fail(ACE_ERR_INVALID_ARG, "null argument");
    *n_pw_half = plan->npw;
    if (miller) std::memcpy(miller, plan->miller.data(), plan->miller.size() * sizeof(int32_t));
    return ACE_OK;
}

int ace_build(ace_plan* plan, const void* psi_G, int n_occ, double alpha, const int32_t* pair_row_ptr,
              const int32_t* pair_col, void* xi, double* E_x, void* stream) {
    if (!plan || !psi_G || !xi) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max) return fail(ACE_ERR_INVALID_ARG, "n_occ out of range");
    if ((pair_row_ptr == nullptr) != (pair_col == nullptr))
        return fail(ACE_ERR_INVALID_ARG, "pair_row_ptr and pair_col must both be set or both be NULL");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->prec == ACE_FP64 ? build_impl<double>(plan, psi_G, n_occ, alpha, pair_row_ptr, pair_col, xi, E_x, st)
                                  : build_impl<float>(plan, psi_G, n_occ, alpha, pair_row_ptr, pair_col, xi, E_x, st);
}

int ace_build_async(ace_plan* plan, const void* psi_G, int n_occ, double alpha, const int32_t* pair_row_ptr,
                    const int32_t* pair_col, void* xi, void* stream) {
    if (!plan || !psi_G || !xi) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max) return fail(ACE_ERR_INVALID_ARG, "n_occ out of range");
    if ((pair_row_ptr == nullptr) != (pair_col == nullptr))
        return fail(ACE_ERR_INVALID_ARG, "pair_row_ptr and pair_col must both be set or both be NULL");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    g_capture = capturing(st);
    const int rc = plan->prec == ACE_FP64
                       ? build_enqueue<double>(plan, psi_G, n_occ, alpha, pair_row_ptr, pair_col, xi, st)
                       : build_enqueue<float>(plan, psi_G, n_occ, alpha, pair_row_ptr, pair_col, xi, st);
    g_capture = false;
    return rc;
}

int ace_build_result(ace_plan* plan, double* E_x, void* stream) {
    if (!plan) return fail(ACE_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(plan->dev);
    return build_finish(plan, E_x, (cudaStream_t)stream);
}

int ace_build_pairs(ace_plan* plan, const void* psi_G, int n_occ, double alpha, const int32_t* pair_row_ptr,
                    const int32_t* pair_col, void* W_G, double* E_part, void* stream) {
    if (!plan || !psi_G || !W_G) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max) return fail(ACE_ERR_INVALID_ARG, "n_occ out of range");
    if ((pair_row_ptr == nullptr) != (pair_col == nullptr))
        return fail(ACE_ERR_INVALID_ARG, "pair_row_ptr and pair_col must both be set or both be NULL");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->prec == ACE_FP64
               ? pairs_impl<double>(plan, psi_G, n_occ, alpha, pair_row_ptr, pair_col, W_G, E_part, st)
               : pairs_impl<float>(plan, psi_G, n_occ, alpha, pair_row_ptr, pair_col, W_G, E_part, st);
}

int ace_overlap_screen(ace_plan* plan, const void* psi_G, int n_occ, double rho_cut, int32_t* pair_row_ptr,
                       int32_t* pair_col, int* n_pairs, double* S, void* stream) {
    if (!plan || !psi_G || !pair_row_ptr || !pair_col) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max) return fail(ACE_ERR_INVALID_ARG, "n_occ out of range");
    if (!(rho_cut >= 0)) return fail(ACE_ERR_INVALID_ARG, "rho_cut must be >= 0");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->prec == ACE_FP64
               ? overlap_impl<double>(plan, psi_G, n_occ, rho_cut, pair_row_ptr, pair_col, n_pairs, S, st)
               : overlap_impl<float>(plan, psi_G, n_occ, rho_cut, pair_row_ptr, pair_col, n_pairs, S, st);
}

int ace_scdm(ace_plan* plan, const void* psi_G, int n_occ, int preselect, void* phi_G, int32_t* pivots,
             int* n_candidates, double* O, void* stream) {
    if (!plan || !psi_G || !phi_G) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max) return fail(ACE_ERR_INVALID_ARG, "n_occ out of range");
    if (n_occ > 2048) return fail(ACE_ERR_INVALID_ARG, "ace_scdm: at most 2048 orbitals");
    const size_t bytes = (size_t)n_occ * plan->npw * 2 * plan->esz;
    const char *a = (const char*)psi_G, *b = (const char*)phi_G;
    if (a < b + bytes && b < a + bytes) return fail(ACE_ERR_INVALID_ARG, "ace_scdm: phi_G overlaps psi_G");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->prec == ACE_FP64
               ? scdm_impl<double>(plan, psi_G, n_occ, preselect, phi_G, pivots, n_candidates, O, st)
               : scdm_impl<float>(plan, psi_G, n_occ, preselect, phi_G, pivots, n_candidates, O, st);
}

int ace_build_finish(ace_plan* plan, const void* psi_G, int n_occ, const void* W_G, void* xi, void* stream) {
    if (!plan || !psi_G || !W_G || !xi) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max) return fail(ACE_ERR_INVALID_ARG, "n_occ out of range");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->prec == ACE_FP64 ? finish_impl<double>(plan, psi_G, n_occ, W_G, xi, st)
                                  : finish_impl<float>(plan, psi_G, n_occ, W_G, xi, st);
}

int ace_apply(ace_plan* plan, const void* xi, int n_occ, const void* psi, int T, void* Kpsi, void* stream) {
    if (!plan || !xi || (T > 0 && (!psi || !Kpsi))) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || T < 0) return fail(ACE_ERR_INVALID_ARG, "n_occ must be >= 1 and T >= 0");
    if (T == 0) return ACE_OK;
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    g_capture = capturing(st);
    const int rc = plan->prec == ACE_FP64 ? apply_impl<double>(plan, xi, n_occ, psi, T, Kpsi, st)
                                          : apply_impl<float>(plan, xi, n_occ, psi, T, Kpsi, st);
    g_capture = false;
    return rc;
}

int ace_apply_prepare(ace_plan* plan, const void* xi, int n_occ, void* stream) {
    if (!plan || !xi) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1) return fail(ACE_ERR_INVALID_ARG, "n_occ must be >= 1");
    plan->ximg_src = nullptr;
    if (plan->prec == ACE_FP64 || !plan->tensor_gram) return ACE_OK;  // nothing to prepare: the product is not split
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    g_capture = capturing(st);
    const long long K = 2LL * plan->npw;
    int rc = grow(&plan->d_ximg, &plan->ximg_cap, xi_image_floats(n_occ, K));
    if (rc == ACE_OK) {
        const cudaError_t e = launch_xi_image((const float*)xi, n_occ, K, plan->d_ximg, st);
        ++plan->launches;
        rc = e == cudaSuccess ? ACE_OK : fail(ACE_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    }
    g_capture = false;
    if (rc == ACE_OK) {
        plan->ximg_src = xi;
        plan->ximg_n = n_occ;
    }
    return rc;
}

int ace_apply_energy(ace_plan* plan, const void* xi, int n_occ, const void* psi, int T, double* E, void* stream) {
    if (!plan || !xi || !E || (T > 0 && !psi)) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || T < 0) return fail(ACE_ERR_INVALID_ARG, "n_occ must be >= 1 and T >= 0");
    *E = 0.0;
    if (T == 0) return ACE_OK;
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    if (capturing(st)) return fail(ACE_ERR_INVALID_ARG, "ace_apply_energy returns a host value and cannot be captured");
    return plan->prec == ACE_FP64 ? apply_energy_impl<double>(plan, xi, n_occ, psi, T, E, st)
                                  : apply_energy_impl<float>(plan, xi, n_occ, psi, T, E, st);
}

int hfx_apply_exact(ace_plan* plan, const void* psi_occ, int n_occ, double alpha, const void* psi, int T,
                    void* Vx_psi, void* stream) {
    if (!plan || !psi_occ || (T > 0 && (!psi || !Vx_psi))) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_occ < 1 || n_occ > plan->n_occ_max || T < 0) return fail(ACE_ERR_INVALID_ARG, "n_occ or T out of range");
    if (T == 0) return ACE_OK;
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    return plan->prec == ACE_FP64 ? hfx_impl<double>(plan, psi_occ, n_occ, alpha, psi, T, Vx_psi, st)
                                  : hfx_impl<float>(plan, psi_occ, n_occ, alpha, psi, T, Vx_psi, st);
}

int ace_build_batched(ace_system* sys, int n_sys, void* stream) {
    if (n_sys < 0 || (n_sys > 0 && !sys)) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (n_sys == 0) return ACE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n_sys; ++i) {
        ace_system& s = sys[i];
        s.E_x = 0;
        s.status = ACE_ERR_INVALID_ARG;
        if (!s.plan || !s.psi_G || !s.xi || s.n_occ < 1 || s.n_occ > s.plan->n_occ_max ||
            (s.pair_row_ptr == nullptr) != (s.pair_col == nullptr))
            return fail(ACE_ERR_INVALID_ARG, "system " + std::to_string(i) + ": invalid arguments");
        if (s.plan->dev != sys[0].plan->dev) return fail(ACE_ERR_INVALID_ARG, "systems on different devices");
        for (int j = 0; j < i; ++j)
            if (sys[j].plan == s.plan) return fail(ACE_ERR_INVALID_ARG, "each system needs its own plan");
    }
    DeviceGuard g(sys[0].plan->dev);
    for (int i = 0; i < n_sys; ++i) {
        ace_system& s = sys[i];
        s.status = s.plan->prec == ACE_FP64 ? check_gamma<double>(s.plan, s.psi_G, s.n_occ, st)
                                            : check_gamma<float>(s.plan, s.psi_G, s.n_occ, st);
        if (s.status != ACE_OK) return s.status;
    }
    // one stream per system, forked from and joined back into the caller's stream
    std::vector<cudaStream_t> ss(n_sys, nullptr);
    std::vector<cudaEvent_t> done(n_sys, nullptr);
    cudaEvent_t fork = nullptr;
    int rc = ACE_OK;
    auto cleanup = [&]() {
        for (auto s : ss)
            if (s) cudaStreamDestroy(s);
        for (auto e : done)
            if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    };
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(fork, st) != cudaSuccess) {
        cleanup();
        return fail(ACE_ERR_CUDA, "event setup failed");
    }
    for (int i = 0; i < n_sys && rc == ACE_OK; ++i) {
        ace_system& s = sys[i];
        if (cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamWaitEvent(ss[i], fork, 0) != cudaSuccess) {
            rc = fail(ACE_ERR_CUDA, "stream setup failed");
            break;
        }
        s.status = s.plan->prec == ACE_FP64
                       ? build_enqueue<double>(s.plan, s.psi_G, s.n_occ, s.alpha, s.pair_row_ptr, s.pair_col, s.xi, ss[i])
                       : build_enqueue<float>(s.plan, s.psi_G, s.n_occ, s.alpha, s.pair_row_ptr, s.pair_col, s.xi, ss[i]);
        if (s.status != ACE_OK) rc = s.status;
        cudaEventRecord(done[i], ss[i]);
    }
    for (int i = 0; i < n_sys; ++i) {
        if (!ss[i]) continue;
        ace_system& s = sys[i];
        if (s.status == ACE_OK) {
            s.status = build_finish(s.plan, &s.E_x, ss[i]);
            if (s.status != ACE_OK && rc == ACE_OK) rc = s.status;
        } else {
            cudaStreamSynchronize(ss[i]);
        }
        cudaStreamWaitEvent(st, done[i], 0);
    }
    cleanup();
    return rc;
}

namespace {
// Version 3 appends the Coulomb cutoff and the G = 0 choice; version 1 files
// (neither field) were written with the bare kernel, G = 0 dropped, and load
// as such; version 2 files carry the cutoff only.
const char kSaveMagic[8] = {'A', 'C', 'E', 'X', 'I', '0', '0', '3'};
const char kSaveMagicV2[8] = {'A', 'C', 'E', 'X', 'I', '0', '0', '2'};
const char kSaveMagicV1[8] = {'A', 'C', 'E', 'X', 'I', '0', '0', '1'};
struct SaveHeader {
    char magic[8];
    int32_t precision, grid[3], n_occ, n_pw_half;
    double cell[9], ecut, alpha, E_x;
    double coulomb_rc;
    int64_t coulomb_g0;
};
constexpr size_t kHeaderV1 = offsetof(SaveHeader, coulomb_rc);
}  // namespace

int ace_save(const char* path, const ace_plan* plan, const void* xi, int n_occ, double alpha, double E_x,
             void* stream) {
    if (!path || !plan || !xi || n_occ < 1 || n_occ > plan->n_occ_max)
        return fail(ACE_ERR_INVALID_ARG, "ace_save: invalid arguments");
    DeviceGuard g(plan->dev);
    const size_t bytes = (size_t)n_occ * plan->npw * 2 * plan->esz;
    std::vector<char> buf(bytes);
    ACE_CK(cudaMemcpyAsync(buf.data(), xi, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    ACE_CK(cudaStreamSynchronize((cudaStream_t)stream));
    SaveHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kSaveMagic, 8);
    h.precision = plan->prec;
    for (int d = 0; d < 3; ++d) h.grid[d] = plan->n[d];
    h.n_occ = n_occ;
    h.n_pw_half = plan->npw;
    std::memcpy(h.cell, plan->cell, sizeof(h.cell));
    h.ecut = plan->ecut;
    h.alpha = alpha;
    h.E_x = E_x;
    h.coulomb_rc = plan->coul_rc;
    h.coulomb_g0 = plan->coul_g0;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(ACE_ERR_INVALID_ARG, std::string("ace_save: cannot open ") + path);
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(buf.data(), 1, bytes, f) == bytes;
    if (std::fclose(f) != 0 || !ok) return fail(ACE_ERR_INVALID_ARG, std::string("ace_save: write failed: ") + path);
    return ACE_OK;
}

int ace_load(const char* path, const ace_plan* plan, void* xi, int* n_occ, double* alpha, double* E_x, void* stream) {
    if (!path || !plan || !xi || !n_occ) return fail(ACE_ERR_INVALID_ARG, "ace_load: invalid arguments");
    plan->ximg_src = nullptr;  // xi's contents change
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ACE_ERR_INVALID_ARG, std::string("ace_load: cannot open ") + path);
    SaveHeader h;
    std::memset(&h, 0, sizeof(h));
    bool hdr = std::fread(&h, kHeaderV1, 1, f) == 1;
    if (hdr && std::memcmp(h.magic, kSaveMagic, 8) == 0)
        hdr = std::fread(&h.coulomb_rc, sizeof(h.coulomb_rc), 1, f) == 1 &&
              std::fread(&h.coulomb_g0, sizeof(h.coulomb_g0), 1, f) == 1;
    else if (hdr && std::memcmp(h.magic, kSaveMagicV2, 8) == 0)
        hdr = std::fread(&h.coulomb_rc, sizeof(h.coulomb_rc), 1, f) == 1;
    else if (hdr)
        hdr = std::memcmp(h.magic, kSaveMagicV1, 8) == 0;
    if (!hdr) {
        std::fclose(f);
        return fail(ACE_ERR_INVALID_ARG, "ace_load: not an ACE vector file");
    }
    bool same = h.precision == plan->prec && h.n_pw_half == plan->npw && h.ecut == plan->ecut &&
                h.coulomb_rc == plan->coul_rc && h.coulomb_g0 == plan->coul_g0;
    for (int d = 0; d < 3; ++d) same = same && h.grid[d] == plan->n[d];
    for (int d = 0; d < 9; ++d) same = same && h.cell[d] == plan->cell[d];
    if (!same || h.n_occ < 1 || h.n_occ > plan->n_occ_max) {
        std::fclose(f);
        return fail(ACE_ERR_INVALID_ARG, "ace_load: file was saved for another grid, cell, cutoff, Coulomb cutoff, precision or size");
    }
    const size_t bytes = (size_t)h.n_occ * plan->npw * 2 * plan->esz;
    std::vector<char> buf(bytes);
    const bool ok = std::fread(buf.data(), 1, bytes, f) == bytes;
    std::fclose(f);
    if (!ok) return fail(ACE_ERR_INVALID_ARG, "ace_load: truncated file");
    DeviceGuard g(plan->dev);
    ACE_CK(cudaMemcpyAsync(xi, buf.data(), bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    ACE_CK(cudaStreamSynchronize((cudaStream_t)stream));
    *n_occ = h.n_occ;
    if (alpha) *alpha = h.alpha;
    if (E_x) *E_x = h.E_x;
    return ACE_OK;
}

int ace_last_intermediates(ace_plan* plan, void* W_G, double* M, void* stream) {
    if (!plan) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (plan->last_n_occ == 0) return fail(ACE_ERR_INVALID_ARG, "no ace_build has run on this plan");
    DeviceGuard g(plan->dev);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = plan->last_n_occ;
    if (W_G)
        ACE_CK(cudaMemcpyAsync(W_G, plan->d_WG, (size_t)n * plan->npw * 2 * plan->esz, cudaMemcpyDeviceToDevice, st));
    if (M) ACE_CK(cudaMemcpyAsync(M, plan->d_M, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    ACE_CK(cudaStreamSynchronize(st));
    return ACE_OK;
}

int ace_check_timeout_path(ace_plan* plan, int limit_ms, void* stream) {
    if (!plan || limit_ms < 1 || limit_ms > 2000) return fail(ACE_ERR_INVALID_ARG, "limit_ms must be 1 .. 2000");
    ace_plan* P = plan;
    DeviceGuard g(P->dev);
    cudaStream_t st = (cudaStream_t)stream;
    ACE_CKL(launch_wait_for_nothing(P->d_err, limit_ms, st));
    ACE_CK(cudaStreamSynchronize(st));
    return check_device_error(P, st);
}

int ace_plan_config(const ace_plan* plan, int* pair_variant, int* pair_streams, float* tune_ms) {
    if (!plan) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (pair_variant) *pair_variant = plan->variant;
    if (pair_streams) *pair_streams = plan->variant == 3 ? 1 : plan->pair_streams;
    if (tune_ms)
        for (int i = 0; i < 6; ++i) tune_ms[i] = plan->tune_ms[i];
    return ACE_OK;
}

int ace_plan_tuning(const ace_plan* plan, int* row_block, float* row_block_ms, int* from_cache) {
    if (!plan) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (row_block) *row_block = plan->row_block;
    if (row_block_ms)
        for (int i = 0; i < 4; ++i) row_block_ms[i] = plan->tune_rb_ms[i];
    if (from_cache) *from_cache = plan->tune_cached;
    return ACE_OK;
}

int ace_plan_radix(const ace_plan* plan, int* radix0, int* n_candidates, int* candidates, float* candidate_ms) {
    if (!plan) return fail(ACE_ERR_INVALID_ARG, "null argument");
    if (radix0) *radix0 = first_radix(plan, plan->pair_r0);
    if (n_candidates) *n_candidates = plan->n_r0_cand;
    for (int k = 0; k < 4; ++k) {
        if (candidates) candidates[k] = k < plan->n_r0_cand ? first_radix(plan, plan->r0_cand[k]) : 0;
        if (candidate_ms) candidate_ms[k] = k < plan->n_r0_cand ? plan->tune_r0_ms[k] : 0.0f;
    }
    return ACE_OK;
}

int ace_set_timing(ace_plan* plan, int enable) {
    if (!plan) return fail(ACE_ERR_INVALID_ARG, "null argument");
    plan->timing = enable != 0;
    return ACE_OK;
}

int ace_get_stats(ace_plan* plan, ace_stats* out) {
    if (!plan || !out) return fail(ACE_ERR_INVALID_ARG, "null argument");
    DeviceGuard g(plan->dev);
    // every timing lane on its own: an interval runs from a mark to the
    // lane's next mark and belongs to the phase of the first
    double ph[PH_N] = {0}, wall = 0, pair_wall = 0;
    auto& mk = plan->marks;
    int lanes = 0;
    for (auto& m : mk) lanes = std::max(lanes, m.lane + 1);
    for (int l = 0; l < lanes; ++l) {
        int prev = -1;
        for (size_t i = 0; i < mk.size(); ++i) {
            if (mk[i].lane != l) continue;
            if (prev >= 0 && mk[prev].phase >= 0) {
                ACE_CK(cudaEventSynchronize(mk[i].ev));
                float ms = 0;
                ACE_CK(cudaEventElapsedTime(&ms, mk[prev].ev, mk[i].ev));
                ph[mk[prev].phase] += ms;
                if (l == 0) wall += ms;
                if (l == 0 && (mk[prev].phase == PH_PAIRWALL || mk[prev].phase == PH_PFWD ||
                               mk[prev].phase == PH_PCOUL || mk[prev].phase == PH_PINV))
                    pair_wall += ms;
            }
            prev = (int)i;
        }
    }
    for (auto& m : mk) ACE_CK(cudaEventSynchronize(m.ev));
    for (auto& m : mk) plan->ev_pool.push_back(m.ev);
    mk.clear();
    std::memset(out, 0, sizeof(*out));
    out->orbitals_ms = ph[PH_ORB];
    out->pair_fwd_ms = ph[PH_PFWD];
    out->pair_coulomb_ms = ph[PH_PCOUL];
    out->pair_inv_ms = ph[PH_PINV];
    out->w_to_g_ms = ph[PH_W2G];
    out->gram_ms = ph[PH_GRAM];
    out->factor_ms = ph[PH_FACTOR];
    out->xi_ms = ph[PH_XI];
    out->energy_ms = ph[PH_ENERGY];
    // wall time of the calls: the intervals of the call's own stream (pair
    // passes spread over pair streams count there as one interval)
    out->total_ms = wall;
    out->pair_wall_ms = pair_wall;
    out->pair_transforms = plan->pair_transforms;
    out->launches = plan->launches;
    plan->pair_transforms = 0;
    plan->launches = 0;
    return ACE_OK;
}

}  // extern "C"

// Record an error for ace_last_error from another translation unit.
int ace::set_last_error(int code, const char* msg) { return fail(code, msg); }

extern "C" {

int ace_last_error(char* buf, int len) {
    const int n = (int)g_err.size();
    if (buf && len > 0) {
        std::strncpy(buf, g_err.c_str(), (size_t)len - 1);
        buf[len - 1] = '\0';
    }
    return n;
}

}  // extern "C"
