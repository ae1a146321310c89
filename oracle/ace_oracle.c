/*
 * ace_oracle.c -- FP64 CPU oracle for the exchange operator and its
 * adaptively compressed (ACE) form, arXiv:2110.07670 Sections 2.1-2.2.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * bench's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only in the seeded
 * inputs of gen/.  Everything here is the plain definition, written out step
 * by step on the discrete grid, in double precision:
 *
 *   psi(r)   = Omega^-1/2 sum_G c(G) e^{iG.r}            (plane-wave expansion)
 *   rho_ij   = phi_i phi_j                               (pair density, Eq. 3)
 *   v_ij     = IFFT[ K(G) FFT(rho_ij) / N ],  K = 4 pi/|G|^2, K(0) = 0
 *   (V_X phi_i)(r) = -alpha sum_j v_ij(r) phi_j(r)       (Eq. 2, scaled by alpha)
 *   E_X      = -alpha sum_{i,j} (Omega/N) sum_r rho_ij v_ij   (Eq. 4)
 *   W = V_X Phi,  M = Phi^T W,  -M = L L^T,  xi = W L^-T   (ACE, Section 2.2)
 *   K psi    = -xi (xi^T psi)                            (Eq. 5)
 *
 * plus a second, independent route to K psi: W M^-1 W^T psi by an LU solve.
 *
 * Readings where the paper is silent (stated again in the design notes):
 * the cutoff is |G|^2 <= ecut[Ry] in bohr^-2 on the half sphere
 * {h>0} U {h=0,k>0} U {h=k=0,l>=0}; the G=0 Coulomb term is dropped; the
 * Coulomb kernel acts on every G of the FFT box (folded to -n/2..n/2-1) with
 * no density-sphere mask; the ACE construction (not printed in the paper) is
 * the standard Cholesky form above.
 *
 * Alternative G=0 treatment (orc_set_coulomb_cutoff): the Coulomb interaction
 * cut off at r = R_c (Spencer & Alavi, Phys. Rev. B 77, 193110 (2008)), whose
 * Fourier transform is K(G) = 4 pi (1 - cos(|G| R_c)) / |G|^2 and
 * K(0) = 2 pi R_c^2; or (orc_set_coulomb_g0) the bare kernel with a given
 * value in place of the dropped G = 0 term (the auxiliary-function
 * correction of Gygi & Baldereschi, computed by the Python side).
 *
 * Parity of every function here is pinned by tests against things other than
 * this file: a brute-force DFT, closed-form Coulomb energies (plane waves and
 * Gaussians), Table 1's plane-wave counts, and invariants of V_X.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#include <unistd.h>

typedef double complex cplx;

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_GRID (-2)
#define ORC_ERR_NOT_POSDEF (-3)
#define ORC_ERR_OOM (-4)
#define ORC_ERR_SINGULAR (-5)

/* ------------------------------------------------------------------ cell */

/* Reciprocal vectors b (rows) with a_i . b_j = 2 pi delta_ij; cell rows are a_i. */
static int reciprocal(const double a[9], double b[9], double *omega)
{
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                 a[2] * (a[3] * a[7] - a[4] * a[6]);
    if (det == 0.0) return ORC_ERR_ARG;
    *omega = fabs(det);
    /* b_i = 2 pi (a_j x a_k) / det */
    const double *a1 = a, *a2 = a + 3, *a3 = a + 6;
    double c[3][3];
    c[0][0] = a2[1] * a3[2] - a2[2] * a3[1];
    c[0][1] = a2[2] * a3[0] - a2[0] * a3[2];
    c[0][2] = a2[0] * a3[1] - a2[1] * a3[0];
    c[1][0] = a3[1] * a1[2] - a3[2] * a1[1];
    c[1][1] = a3[2] * a1[0] - a3[0] * a1[2];
    c[1][2] = a3[0] * a1[1] - a3[1] * a1[0];
    c[2][0] = a1[1] * a2[2] - a1[2] * a2[1];
    c[2][1] = a1[2] * a2[0] - a1[0] * a2[2];
    c[2][2] = a1[0] * a2[1] - a1[1] * a2[0];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b[3 * i + j] = 2.0 * M_PI * c[i][j] / det;
    return ORC_OK;
}

static void gvec(const double b[9], int h, int k, int l, double g[3])
{
    for (int j = 0; j < 3; ++j) g[j] = h * b[j] + k * b[3 + j] + l * b[6 + j];
}

/*
 * Half sphere of plane waves, |G|^2 <= ecut_ry (Table 1 convention), in
 * lexicographic (h,k,l) order over {h>0} U {h=0,k>0} U {h=k=0,l>=0}.
 * Writes up to cap Miller triples; returns the count in *n_out.
 */
int orc_half_sphere(const double cell[9], double ecut_ry, int cap, int32_t *miller, int *n_out)
{
    double b[9], omega;
    if (reciprocal(cell, b, &omega) != ORC_OK || ecut_ry <= 0) return ORC_ERR_ARG;
    int lim[3];
    for (int i = 0; i < 3; ++i) {
        double len = sqrt(cell[3 * i] * cell[3 * i] + cell[3 * i + 1] * cell[3 * i + 1] +
                          cell[3 * i + 2] * cell[3 * i + 2]);
        lim[i] = (int)floor(sqrt(ecut_ry) * len / (2.0 * M_PI)) + 1;
    }
    int n = 0;
    for (int h = 0; h <= lim[0]; ++h)
        for (int k = -lim[1]; k <= lim[1]; ++k)
            for (int l = -lim[2]; l <= lim[2]; ++l) {
                if (!(h > 0 || (h == 0 && k > 0) || (h == 0 && k == 0 && l >= 0))) continue;
                double g[3];
                gvec(b, h, k, l, g);
                if (g[0] * g[0] + g[1] * g[1] + g[2] * g[2] > ecut_ry) continue;
                if (miller && n < cap) {
                    miller[3 * n] = h;
                    miller[3 * n + 1] = k;
                    miller[3 * n + 2] = l;
                }
                ++n;
            }
    *n_out = n;
    return ORC_OK;
}

/* ------------------------------------------------------------------- FFT */

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * Recursive mixed-radix decimation-in-time Cooley-Tukey DFT:
 *   X[k] = sum_j x[j] w^{jk},  w = exp(sign 2 pi i / n).
 * With n = p m and x split by residue r = j mod p into p DFTs Y_r of size m,
 *   X[k + m s] = sum_r w_n^{r k} w_p^{r s} Y_r[k].
 * tw[t * tstride] = exp(sign 2 pi i t / n) for t < n.
 */
static void fft1d_rec(const cplx *in, int istride, cplx *out, int n, const cplx *tw, int tstride)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int p = smallest_factor(n), m = n / p;
    for (int r = 0; r < p; ++r) fft1d_rec(in + r * istride, istride * p, out + r * m, m, tw, tstride * p);
    cplx *t = malloc(sizeof(cplx) * p);
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) t[r] = out[r * m + k] * tw[(int)(((long)r * k) % n) * tstride];
        for (int s = 0; s < p; ++s) {
            cplx acc = 0;
            for (int r = 0; r < p; ++r) acc += t[r] * tw[(int)(((long)r * s * m) % n) * tstride];
            out[s * m + k] = acc;
        }
    }
    free(t);
}

/* In-place 3D DFT of a [n0][n1][n2] row-major complex array (unnormalised). */
void orc_fft3d(cplx *a, const int n[3], int sign)
{
    int nmax = n[0] > n[1] ? n[0] : n[1];
    if (n[2] > nmax) nmax = n[2];
    cplx *line = malloc(sizeof(cplx) * nmax), *out = malloc(sizeof(cplx) * nmax);
    cplx *tw = malloc(sizeof(cplx) * nmax);
    long s[3] = {(long)n[1] * n[2], n[2], 1};
    for (int ax = 0; ax < 3; ++ax) {
        int len = n[ax];
        for (int t = 0; t < len; ++t) tw[t] = cexp(sign * 2.0 * M_PI * I * (double)t / len);
        int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
        for (int i1 = 0; i1 < n[o1]; ++i1)
            for (int i2 = 0; i2 < n[o2]; ++i2) {
                cplx *base = a + i1 * s[o1] + i2 * s[o2];
                for (int t = 0; t < len; ++t) line[t] = base[t * s[ax]];
                fft1d_rec(line, 1, out, len, tw, 1);
                for (int t = 0; t < len; ++t) base[t * s[ax]] = out[t];
            }
    }
    free(line);
    free(out);
    free(tw);
}

/* ------------------------------------------------------- grid / Coulomb */

typedef struct {
    int n[3];
    long N;
    double b[9], omega;
    int npw;
    const int32_t *miller;
} grid_t;

static int fold(int i, int n) { return i < n - n / 2 ? i : i - n; } /* 0..n-1 -> -n/2..n/2-1 */
static int wrap(int m, int n) { return ((m % n) + n) % n; }

static int grid_init(grid_t *g, const int n[3], const double cell[9], int npw, const int32_t *miller)
{
    if (reciprocal(cell, g->b, &g->omega) != ORC_OK) return ORC_ERR_ARG;
    for (int i = 0; i < 3; ++i) g->n[i] = n[i];
    g->N = (long)n[0] * n[1] * n[2];
    g->npw = npw;
    g->miller = miller;
    for (int p = 0; p < npw; ++p)
        for (int i = 0; i < 3; ++i)
            if (2 * abs(miller[3 * p + i]) + 1 > n[i]) return ORC_ERR_GRID;
    return ORC_OK;
}

static long box_index(const grid_t *g, int h, int k, int l)
{
    return ((long)wrap(h, g->n[0]) * g->n[1] + wrap(k, g->n[1])) * g->n[2] + wrap(l, g->n[2]);
}

/* Truncation radius of the Coulomb interaction; 0: the bare 1/r with G = 0 dropped. */
static double coulomb_rc = 0.0;

void orc_set_coulomb_cutoff(double rc) { coulomb_rc = rc > 0.0 ? rc : 0.0; }

/* K(0) of the bare kernel (0: the G = 0 term dropped). */
static double coulomb_k0 = 0.0;

void orc_set_coulomb_g0(double k0) { coulomb_k0 = k0; }

/* Coulomb kernel for box entry (i0,i1,i2): 4 pi / |G|^2 with G = 0 dropped,
 * or, with a cutoff R_c, the transform of 1/r restricted to r < R_c. */
static double coulomb(const grid_t *g, int i0, int i1, int i2)
{
    double G[3];
    gvec(g->b, fold(i0, g->n[0]), fold(i1, g->n[1]), fold(i2, g->n[2]), G);
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    if (coulomb_rc > 0.0)
        return g2 == 0.0 ? 2.0 * M_PI * coulomb_rc * coulomb_rc
                         : 4.0 * M_PI * (1.0 - cos(sqrt(g2) * coulomb_rc)) / g2;
    return g2 == 0.0 ? coulomb_k0 : 4.0 * M_PI / g2;
}

/* psi(r) on the grid from half-sphere coefficients: full sphere via c(-G) = c(G)^*. */
static void to_real(const grid_t *g, const cplx *c, cplx *box, double *out)
{
    memset(box, 0, sizeof(cplx) * g->N);
    for (int p = 0; p < g->npw; ++p) {
        const int32_t *m = g->miller + 3 * p;
        box[box_index(g, m[0], m[1], m[2])] = c[p];
        if (m[0] || m[1] || m[2]) box[box_index(g, -m[0], -m[1], -m[2])] = conj(c[p]);
    }
    orc_fft3d(box, g->n, +1);
    double s = 1.0 / sqrt(g->omega);
    for (long r = 0; r < g->N; ++r) out[r] = creal(box[r]) * s;
}

/* Half-sphere coefficients of a real grid function f: Omega^1/2 / N FFT(f). */
static void to_recip(const grid_t *g, const double *f, cplx *box, cplx *c)
{
    for (long r = 0; r < g->N; ++r) box[r] = f[r];
    orc_fft3d(box, g->n, -1);
    double s = sqrt(g->omega) / (double)g->N;
    for (int p = 0; p < g->npw; ++p) {
        const int32_t *m = g->miller + 3 * p;
        c[p] = box[box_index(g, m[0], m[1], m[2])] * s;
    }
}

/* v = IFFT[K FFT(rho)/N] for a real rho (Eq. 3 solved in reciprocal space). */
static void poisson(const grid_t *g, const double *rho, cplx *box, double *v)
{
    for (long r = 0; r < g->N; ++r) box[r] = rho[r];
    orc_fft3d(box, g->n, -1);
    long q = 0;
    for (int i0 = 0; i0 < g->n[0]; ++i0)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i2 = 0; i2 < g->n[2]; ++i2, ++q) box[q] *= coulomb(g, i0, i1, i2) / (double)g->N;
    orc_fft3d(box, g->n, +1);
    for (long r = 0; r < g->N; ++r) v[r] = creal(box[r]);
}

/* <a|b> of two real functions given on the half sphere, summed over the full sphere. */
static double gamma_dot(const grid_t *g, const cplx *a, const cplx *b)
{
    cplx s = 0;
    for (int p = 0; p < g->npw; ++p) {
        const int32_t *m = g->miller + 3 * p;
        s += conj(a[p]) * b[p];                         /* +G */
        if (m[0] || m[1] || m[2]) s += a[p] * conj(b[p]); /* -G: conj(conj a) conj b */
    }
    return creal(s);
}

static int check_gamma(int npw, const int32_t *miller, const cplx *c, int n)
{
    (void)npw;
    if (miller[0] || miller[1] || miller[2]) return ORC_OK;
    for (int i = 0; i < n; ++i)
        if (fabs(cimag(c[(long)i * npw])) > 1e-6) return ORC_ERR_ARG;
    return ORC_OK;
}

/* --------------------------------------------------- exchange (Eq. 2-4) */

/*
 * Work list: "left" functions f_a (a < n_left) and "right" orbitals phi_b.
 * For every listed pair (a,b): v = Poisson(f_a phi_b);
 *   acc_left[a]  += v phi_b;
 *   if symmetric and the pair is off-diagonal: acc_right[b] += v f_a;
 *   e_sum += (2 - delta_ab) (Omega/N) sum_r f_a phi_b v   (symmetric only).
 * Pairs are split over threads; each accumulator row has its own lock.
 */
typedef struct {
    const grid_t *g;
    const double *left, *right; /* [n][N] */
    double *acc_left, *acc_right;
    int symmetric;
    const int32_t *pa, *pb;
    long npairs;
    pthread_mutex_t *lock_left, *lock_right;
    long next;
    pthread_mutex_t next_lock;
    double e_sum;
    pthread_mutex_t e_lock;
} xwork_t;

static void *xworker(void *arg)
{
    xwork_t *w = arg;
    const grid_t *g = w->g;
    long N = g->N;
    double *rho = malloc(sizeof(double) * N), *v = malloc(sizeof(double) * N);
    double *tmp = malloc(sizeof(double) * N);
    cplx *box = malloc(sizeof(cplx) * N);
    for (;;) {
        pthread_mutex_lock(&w->next_lock);
        long q = w->next++;
        pthread_mutex_unlock(&w->next_lock);
        if (q >= w->npairs) break;
        int a = w->pa[q], b = w->pb[q];
        const double *fa = w->left + (long)a * N, *fb = w->right + (long)b * N;
        for (long r = 0; r < N; ++r) rho[r] = fa[r] * fb[r];
        poisson(g, rho, box, v);
        double e = 0;
        for (long r = 0; r < N; ++r) e += rho[r] * v[r];
        e *= g->omega / (double)N;
        for (long r = 0; r < N; ++r) tmp[r] = v[r] * fb[r];
        pthread_mutex_lock(&w->lock_left[a]);
        double *dl = w->acc_left + (long)a * N;
        for (long r = 0; r < N; ++r) dl[r] += tmp[r];
        pthread_mutex_unlock(&w->lock_left[a]);
        int offdiag = !(w->symmetric && a == b);
        if (w->symmetric && offdiag) {
            for (long r = 0; r < N; ++r) tmp[r] = v[r] * fa[r];
            pthread_mutex_lock(&w->lock_right[b]);
            double *dr = w->acc_right + (long)b * N;
            for (long r = 0; r < N; ++r) dr[r] += tmp[r];
            pthread_mutex_unlock(&w->lock_right[b]);
        }
        pthread_mutex_lock(&w->e_lock);
        w->e_sum += (offdiag ? 2.0 : 1.0) * e;
        pthread_mutex_unlock(&w->e_lock);
    }
    free(rho);
    free(v);
    free(tmp);
    free(box);
    return NULL;
}

static int run_pairs(xwork_t *w, int nthreads)
{
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    pthread_mutex_init(&w->next_lock, NULL);
    pthread_mutex_init(&w->e_lock, NULL);
    w->next = 0;
    w->e_sum = 0;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, xworker, w);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&w->next_lock);
    pthread_mutex_destroy(&w->e_lock);
    return ORC_OK;
}

static pthread_mutex_t *new_locks(int n)
{
    pthread_mutex_t *l = malloc(sizeof(pthread_mutex_t) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) pthread_mutex_init(&l[i], NULL);
    return l;
}

static void free_locks(pthread_mutex_t *l, int n)
{
    for (int i = 0; i < n; ++i) pthread_mutex_destroy(&l[i]);
    free(l);
}

/* Run fn(ctx, i, scratch) for i < n over nthreads threads (static round robin). */
typedef struct {
    void (*fn)(void *, int, cplx *);
    void *ctx;
    int n, nt, tid;
    long scratch;
} pfor_t;

static void *pfor_worker(void *arg)
{
    pfor_t *p = arg;
    cplx *scratch = malloc(sizeof(cplx) * p->scratch);
    for (int i = p->tid; i < p->n; i += p->nt) p->fn(p->ctx, i, scratch);
    free(scratch);
    return NULL;
}

static void parallel_for(int n, int nthreads, long scratch, void (*fn)(void *, int, cplx *), void *ctx)
{
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    pfor_t *args = malloc(sizeof(pfor_t) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        args[t] = (pfor_t){fn, ctx, n, nthreads, t, scratch};
        pthread_create(&th[t], NULL, pfor_worker, &args[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(args);
}

typedef struct {
    const grid_t *g;
    const cplx *c;
    double *f;
    cplx *cout;
    double scale;
} map_t;

static void to_real_one(void *ctx, int i, cplx *box)
{
    map_t *m = ctx;
    to_real(m->g, m->c + (long)i * m->g->npw, box, m->f + (long)i * m->g->N);
}

static void to_recip_one(void *ctx, int i, cplx *box)
{
    map_t *m = ctx;
    double *f = m->f + (long)i * m->g->N;
    for (long r = 0; r < m->g->N; ++r) f[r] *= m->scale;
    to_recip(m->g, f, box, m->cout + (long)i * m->g->npw);
}

typedef struct {
    const grid_t *g;
    const cplx *c;
    double *f;
    const int32_t *list;
} listmap_t;

static void to_real_listed(void *ctx, int q, cplx *box)
{
    listmap_t *m = ctx;
    int i = m->list[q];
    to_real(m->g, m->c + (long)i * m->g->npw, box, m->f + (long)i * m->g->N);
}

static double wall(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* Expand a CSR list (row i: cols j >= i), or every i <= j when row_ptr is NULL. */
static long expand_pairs(int n, const int32_t *row_ptr, const int32_t *col, int32_t **pa, int32_t **pb)
{
    long np = row_ptr ? row_ptr[n] : (long)n * (n + 1) / 2;
    *pa = malloc(sizeof(int32_t) * (np > 0 ? np : 1));
    *pb = malloc(sizeof(int32_t) * (np > 0 ? np : 1));
    long q = 0;
    for (int i = 0; i < n; ++i) {
        if (row_ptr) {
            for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t, ++q) {
                (*pa)[q] = i;
                (*pb)[q] = col[t];
            }
        } else {
            for (int j = i; j < n; ++j, ++q) {
                (*pa)[q] = i;
                (*pb)[q] = j;
            }
        }
    }
    return np;
}

/*
 * Exchange of the occupied set with itself (Eq. 2 and 4), restricted to the
 * listed pairs: W_G[i] = half-sphere coefficients of (V_X phi_i), scaled by
 * alpha, and E_X = -alpha sum (2 - delta_ij) e_ij.  times (may be NULL)
 * receives the wall seconds of the orbital transforms, the pair solves and
 * the back transforms.
 */
int orc_exchange_timed(const double *psi_G, int n_occ, int npw, const int32_t *miller, const int grid[3],
                       const double cell[9], double alpha, const int32_t *row_ptr, const int32_t *col,
                       int nthreads, double *W_G, double *E_x, double *times);

int orc_exchange(const double *psi_G, int n_occ, int npw, const int32_t *miller, const int grid[3],
                 const double cell[9], double alpha, const int32_t *row_ptr, const int32_t *col,
                 int nthreads, double *W_G, double *E_x)
{
    return orc_exchange_timed(psi_G, n_occ, npw, miller, grid, cell, alpha, row_ptr, col, nthreads, W_G, E_x, NULL);
}

int orc_exchange_timed(const double *psi_G, int n_occ, int npw, const int32_t *miller, const int grid[3],
                       const double cell[9], double alpha, const int32_t *row_ptr, const int32_t *col,
                       int nthreads, double *W_G, double *E_x, double *times)
{
    grid_t g;
    int st = grid_init(&g, grid, cell, npw, miller);
    if (st) return st;
    if (n_occ < 1) return ORC_ERR_ARG;
    const cplx *c = (const cplx *)psi_G;
    if ((st = check_gamma(npw, miller, c, n_occ))) return st;
    long N = g.N;
    double *phi = malloc(sizeof(double) * N * n_occ), *acc = calloc((size_t)N * n_occ, sizeof(double));
    cplx *box = malloc(sizeof(cplx) * N);
    if (!phi || !acc || !box) return ORC_ERR_OOM;
    double t0 = wall();
    map_t mp = {.g = &g, .c = c, .f = phi};
    parallel_for(n_occ, nthreads, N, to_real_one, &mp);
    double t1 = wall();
    int32_t *pa, *pb;
    long np = expand_pairs(n_occ, row_ptr, col, &pa, &pb);
    pthread_mutex_t *locks = new_locks(n_occ);
    xwork_t w = {.g = &g, .left = phi, .right = phi, .acc_left = acc, .acc_right = acc, .symmetric = 1,
                 .pa = pa, .pb = pb, .npairs = np, .lock_left = locks, .lock_right = locks};
    run_pairs(&w, nthreads);
    double t2 = wall();
    free_locks(locks, n_occ);
    free(pa);
    free(pb);
    if (E_x) *E_x = -alpha * w.e_sum;
    if (W_G) {
        map_t mb = {.g = &g, .f = acc, .cout = (cplx *)W_G, .scale = -alpha};
        parallel_for(n_occ, nthreads, N, to_recip_one, &mb);
    }
    if (times) {
        times[0] = t1 - t0;
        times[1] = t2 - t1;
        times[2] = wall() - t2;
    }
    free(phi);
    free(acc);
    free(box);
    return ORC_OK;
}

/*
 * Rows of the (possibly screened) exchange: for each requested orbital i,
 * W_G[i] = -alpha sum_{j : (min(i,j), max(i,j)) listed} v_ij phi_j on the half
 * sphere (Eq. 2 restricted to the kept pairs), the same quantity as row i of
 * orc_exchange's W_G, computed from the orbitals those rows need only.
 * row_ptr/col: CSR of kept pairs i <= j, or NULL for every pair.
 */
int orc_exchange_rows(const double *psi_G, int n_occ, int npw, const int32_t *miller, const int grid[3],
                      const double cell[9], double alpha, const int32_t *row_ptr, const int32_t *col, int nrows,
                      const int32_t *rows, int nthreads, double *W_rows)
{
    grid_t g;
    int st = grid_init(&g, grid, cell, npw, miller);
    if (st) return st;
    if (n_occ < 1 || nrows < 1) return ORC_ERR_ARG;
    for (int k = 0; k < nrows; ++k)
        if (rows[k] < 0 || rows[k] >= n_occ) return ORC_ERR_ARG;
    long N = g.N;
    /* pairs (row k, orbital j) with (min, max) in the list */
    int32_t *pa = malloc(sizeof(int32_t) * (long)nrows * n_occ), *pb = malloc(sizeof(int32_t) * (long)nrows * n_occ);
    char *need = calloc(n_occ, 1);
    long np = 0;
    for (int k = 0; k < nrows; ++k) {
        int i = rows[k];
        need[i] = 1;
        for (int j = 0; j < n_occ; ++j) {
            int lo = i < j ? i : j, hi = i < j ? j : i, kept = 1;
            if (row_ptr) {
                kept = 0;
                for (int32_t t = row_ptr[lo]; t < row_ptr[lo + 1]; ++t)
                    if (col[t] == hi) kept = 1;
            }
            if (kept) {
                pa[np] = k;
                pb[np] = j;
                need[j] = 1;
                ++np;
            }
        }
    }
    /* real-space orbitals: only those the rows touch (others stay zero) */
    double *phi = calloc((size_t)N * n_occ, sizeof(double)), *f = malloc(sizeof(double) * N * nrows);
    double *acc = calloc((size_t)N * nrows, sizeof(double));
    int nneed = 0;
    for (int j = 0; j < n_occ; ++j) nneed += need[j];
    int32_t *list = malloc(sizeof(int32_t) * (nneed > 0 ? nneed : 1));
    for (int j = 0, q = 0; j < n_occ; ++j)
        if (need[j]) list[q++] = j;
    cplx *box = malloc(sizeof(cplx) * N);
    listmap_t lm = {.g = &g, .c = (const cplx *)psi_G, .f = phi, .list = list};
    parallel_for(nneed, nthreads, N, to_real_listed, &lm);
    for (int k = 0; k < nrows; ++k) memcpy(f + (long)k * N, phi + (long)rows[k] * N, sizeof(double) * N);
    pthread_mutex_t *locks = new_locks(nrows);
    xwork_t w = {.g = &g, .left = f, .right = phi, .acc_left = acc, .acc_right = NULL, .symmetric = 0,
                 .pa = pa, .pb = pb, .npairs = np, .lock_left = locks, .lock_right = NULL};
    run_pairs(&w, nthreads);
    free_locks(locks, nrows);
    map_t m = {.g = &g, .f = acc, .cout = (cplx *)W_rows, .scale = -alpha};
    parallel_for(nrows, nthreads, N, to_recip_one, &m);
    free(pa);
    free(pb);
    free(need);
    free(list);
    free(phi);
    free(f);
    free(acc);
    free(box);
    return ORC_OK;
}

/* V_X psi_t for trial vectors (Eq. 2 over all occupied j), scaled by alpha. */
int orc_vx_apply(const double *psi_occ, int n_occ, const double *psi_trial, int T, int npw,
                 const int32_t *miller, const int grid[3], const double cell[9], double alpha, int nthreads,
                 double *out)
{
    grid_t g;
    int st = grid_init(&g, grid, cell, npw, miller);
    if (st) return st;
    if (n_occ < 1 || T < 0) return ORC_ERR_ARG;
    if (T == 0) return ORC_OK;
    long N = g.N;
    double *phi = malloc(sizeof(double) * N * n_occ), *f = malloc(sizeof(double) * N * T);
    double *acc = calloc((size_t)N * T, sizeof(double));
    cplx *box = malloc(sizeof(cplx) * N);
    if (!phi || !f || !acc || !box) return ORC_ERR_OOM;
    map_t m1 = {.g = &g, .c = (const cplx *)psi_occ, .f = phi};
    parallel_for(n_occ, nthreads, N, to_real_one, &m1);
    map_t m2 = {.g = &g, .c = (const cplx *)psi_trial, .f = f};
    parallel_for(T, nthreads, N, to_real_one, &m2);
    long np = (long)T * n_occ;
    int32_t *pa = malloc(sizeof(int32_t) * np), *pb = malloc(sizeof(int32_t) * np);
    for (long q = 0; q < np; ++q) {
        pa[q] = (int32_t)(q / n_occ);
        pb[q] = (int32_t)(q % n_occ);
    }
    pthread_mutex_t *locks = new_locks(T);
    xwork_t w = {.g = &g, .left = f, .right = phi, .acc_left = acc, .acc_right = NULL, .symmetric = 0,
                 .pa = pa, .pb = pb, .npairs = np, .lock_left = locks, .lock_right = NULL};
    run_pairs(&w, nthreads);
    free_locks(locks, T);
    map_t m3 = {.g = &g, .f = acc, .cout = (cplx *)out, .scale = -alpha};
    parallel_for(T, nthreads, N, to_recip_one, &m3);
    free(pa);
    free(pb);
    free(phi);
    free(f);
    free(acc);
    free(box);
    return ORC_OK;
}

/* Coulomb pair energy e_ab = (Omega/N) sum_r rho_ab v_ab of two orbitals (Eq. 4 term). */
int orc_pair_energy(const double *c_a, const double *c_b, int npw, const int32_t *miller, const int grid[3],
                    const double cell[9], double *e)
{
    grid_t g;
    int st = grid_init(&g, grid, cell, npw, miller);
    if (st) return st;
    long N = g.N;
    double *fa = malloc(sizeof(double) * N), *fb = malloc(sizeof(double) * N);
    double *rho = malloc(sizeof(double) * N), *v = malloc(sizeof(double) * N);
    cplx *box = malloc(sizeof(cplx) * N);
    to_real(&g, (const cplx *)c_a, box, fa);
    to_real(&g, (const cplx *)c_b, box, fb);
    for (long r = 0; r < N; ++r) rho[r] = fa[r] * fb[r];
    poisson(&g, rho, box, v);
    double s = 0;
    for (long r = 0; r < N; ++r) s += rho[r] * v[r];
    *e = s * g.omega / (double)N;
    free(fa);
    free(fb);
    free(rho);
    free(v);
    free(box);
    return ORC_OK;
}

/* Orbitals on the real-space grid, [n][N] doubles. */
int orc_to_real(const double *psi_G, int n, int npw, const int32_t *miller, const int grid[3],
                const double cell[9], double *out)
{
    grid_t g;
    int st = grid_init(&g, grid, cell, npw, miller);
    if (st) return st;
    cplx *box = malloc(sizeof(cplx) * g.N);
    for (int i = 0; i < n; ++i) to_real(&g, (const cplx *)psi_G + (long)i * npw, box, out + (long)i * g.N);
    free(box);
    return ORC_OK;
}

/* Orbital overlap of the s-MTACE screening (Section 2.4):
 *   S_ij = integral |phi_i(r) phi_j(r)| dr = (Omega / N) sum_r |phi_i(r)| |phi_j(r)|
 * on the real-space grid, for every i, j (S is n x n, row-major; computed for
 * i <= j and mirrored). */
int orc_overlap(const double *psi_G, int n, int npw, const int32_t *miller, const int grid[3], const double cell[9],
                double *S)
{
    grid_t g;
    int st = grid_init(&g, grid, cell, npw, miller);
    if (st) return st;
    double *f = malloc(sizeof(double) * (size_t)n * g.N);
    cplx *box = malloc(sizeof(cplx) * g.N);
    if (!f || !box) {
        free(f);
        free(box);
        return ORC_ERR_OOM;
    }
    for (int i = 0; i < n; ++i) to_real(&g, (const cplx *)psi_G + (long)i * npw, box, f + (long)i * g.N);
    const double dv = g.omega / (double)g.N;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            const double *a = f + (long)i * g.N, *b = f + (long)j * g.N;
            double sum = 0.0;
            for (long r = 0; r < g.N; ++r) sum += fabs(a[r] * b[r]);
            S[(long)i * n + j] = S[(long)j * n + i] = sum * dv;
        }
    free(f);
    free(box);
    return ORC_OK;
}

/* ------------------------------------------------------ ACE (Section 2.2) */

/* Gram matrix G_ij = <a_i|b_j> (full-sphere inner product of real functions). */
int orc_gamma_gram(const double *a, int na, const double *b, int nb, int npw, const int32_t *miller,
                   double *out)
{
    grid_t g = {.npw = npw, .miller = miller};
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
            out[(long)i * nb + j] =
                gamma_dot(&g, (const cplx *)a + (long)i * npw, (const cplx *)b + (long)j * npw);
    return ORC_OK;
}

/* Cholesky A = L L^T of a symmetric positive definite n x n matrix (row-major). */
int orc_cholesky(const double *A, int n, double *L)
{
    memset(L, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[(long)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(long)i * n + k] * L[(long)j * n + k];
            if (i == j) {
                if (!(s > 0)) return ORC_ERR_NOT_POSDEF;
                L[(long)i * n + i] = sqrt(s);
            } else {
                L[(long)i * n + j] = s / L[(long)j * n + j];
            }
        }
    return ORC_OK;
}

/*
 * ACE build: W = V_X Phi (alpha-scaled), M = Phi^T W, -M = L L^T,
 * xi = W L^-T, i.e. row k of xi solves sum_{m<=k} L_km xi_m = W_k.
 * Then K = -xi xi^T = W M^-1 W^T reproduces V_X on span(Phi).
 * Optional outputs W_G_out [n_occ][npw] and M_out [n_occ][n_occ] may be NULL.
 */
int orc_ace_build(const double *psi_G, int n_occ, int npw, const int32_t *miller, const int grid[3],
                  const double cell[9], double alpha, const int32_t *row_ptr, const int32_t *col, int nthreads,
                  double *xi, double *E_x, double *W_G_out, double *M_out)
{
    long sz = (long)n_occ * npw;
    cplx *W = malloc(sizeof(cplx) * sz);
    double *M = malloc(sizeof(double) * n_occ * n_occ), *L = malloc(sizeof(double) * n_occ * n_occ);
    int st = orc_exchange(psi_G, n_occ, npw, miller, grid, cell, alpha, row_ptr, col, nthreads, (double *)W, E_x);
    if (st) goto done;
    orc_gamma_gram(psi_G, n_occ, (const double *)W, n_occ, npw, miller, M);
    if (M_out) memcpy(M_out, M, sizeof(double) * n_occ * n_occ);
    if (W_G_out) memcpy(W_G_out, W, sizeof(cplx) * sz);
    for (long q = 0; q < (long)n_occ * n_occ; ++q) M[q] = -M[q];
    /* symmetrise -M before factoring: M is symmetric up to rounding */
    for (int i = 0; i < n_occ; ++i)
        for (int j = 0; j < i; ++j) {
            double s = 0.5 * (M[(long)i * n_occ + j] + M[(long)j * n_occ + i]);
            M[(long)i * n_occ + j] = M[(long)j * n_occ + i] = s;
        }
    if ((st = orc_cholesky(M, n_occ, L))) goto done;
    cplx *X = (cplx *)xi;
    for (int k = 0; k < n_occ; ++k)
        for (int p = 0; p < npw; ++p) {
            cplx s = W[(long)k * npw + p];
            for (int m = 0; m < k; ++m) s -= L[(long)k * n_occ + m] * X[(long)m * npw + p];
            X[(long)k * npw + p] = s / L[(long)k * n_occ + k];
        }
done:
    free(W);
    free(M);
    free(L);
    return st;
}

/* K psi = -xi (xi^T psi) (Eq. 5 with P = xi). */
int orc_ace_apply(const double *xi, int n_occ, const double *psi, int T, int npw, const int32_t *miller,
                  double *out)
{
    double *C = malloc(sizeof(double) * ((long)n_occ * T + 1));
    orc_gamma_gram(xi, n_occ, psi, T, npw, miller, C); /* C_kt = <xi_k|psi_t> */
    const cplx *X = (const cplx *)xi;
    cplx *O = (cplx *)out;
    for (int t = 0; t < T; ++t)
        for (int p = 0; p < npw; ++p) {
            cplx s = 0;
            for (int k = 0; k < n_occ; ++k) s += X[(long)k * npw + p] * C[(long)k * T + t];
            O[(long)t * npw + p] = -s;
        }
    free(C);
    return ORC_OK;
}

/*
 * Second route to the same operator: K psi = W M^-1 (W^T psi), solving
 * M X = B by Gaussian elimination with partial pivoting.  It shares nothing
 * with the Cholesky route above except the inputs W and M.
 */
int orc_ace_apply_lu(const double *W_G, const double *M_in, int n_occ, const double *psi, int T, int npw,
                     const int32_t *miller, double *out)
{
    int n = n_occ;
    double *A = malloc(sizeof(double) * n * n), *B = malloc(sizeof(double) * ((long)n * T + 1));
    memcpy(A, M_in, sizeof(double) * n * n);
    orc_gamma_gram(W_G, n, psi, T, npw, miller, B); /* B_kt = <W_k|psi_t> */
    int st = ORC_OK;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[(long)r * n + c]) > fabs(A[(long)piv * n + c])) piv = r;
        if (A[(long)piv * n + c] == 0.0) {
            st = ORC_ERR_SINGULAR;
            goto done;
        }
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[(long)c * n + k];
                A[(long)c * n + k] = A[(long)piv * n + k];
                A[(long)piv * n + k] = t;
            }
            for (int k = 0; k < T; ++k) {
                double t = B[(long)c * T + k];
                B[(long)c * T + k] = B[(long)piv * T + k];
                B[(long)piv * T + k] = t;
            }
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[(long)r * n + c] / A[(long)c * n + c];
            for (int k = c; k < n; ++k) A[(long)r * n + k] -= f * A[(long)c * n + k];
            for (int k = 0; k < T; ++k) B[(long)r * T + k] -= f * B[(long)c * T + k];
        }
    }
    for (int c = n - 1; c >= 0; --c)
        for (int k = 0; k < T; ++k) {
            double s = B[(long)c * T + k];
            for (int m = c + 1; m < n; ++m) s -= A[(long)c * n + m] * B[(long)m * T + k];
            B[(long)c * T + k] = s / A[(long)c * n + c];
        }
    {
        const cplx *Wc = (const cplx *)W_G;
        cplx *O = (cplx *)out;
        for (int t = 0; t < T; ++t)
            for (int p = 0; p < npw; ++p) {
                cplx s = 0;
                for (int k = 0; k < n; ++k) s += Wc[(long)k * npw + p] * B[(long)k * T + t];
                O[(long)t * npw + p] = s;
            }
    }
done:
    free(A);
    free(B);
    return st;
}
