// fft_core.cuh -- complex arithmetic, radix-2/3/4/5/8 DFT codelets and the
// in-place mixed-radix stages of the library's batched 1D transforms.
//
// The pair Poisson solves of the exchange operator (arXiv:2110.07670 Section
// 2.1, Eq. 3, evaluated in reciprocal space as the paper describes) are 3D
// FFTs; every pass kernel of this library is built from the stages below.
//
// Forward transform, decimation in frequency, in place.  With radices
// r_1 .. r_m (product n), stage i works on blocks of length L_i = n / (r_1 ..
// r_{i-1}) with m_i = L_i / r_i.  Butterfly (block beta, j < m_i) reads the
// r_i elements at beta L_i + j + m_i q, forms
//     y_s = w_{L_i}^{j s} sum_q x_q w_{r_i}^{q s},   w_L = exp(-2 pi i / L),
// and writes y_s back to beta L_i + j + m_i s.  Frequency k with mixed-radix
// digits k = s_1 + r_1 (s_2 + r_2 (s_3 + ...)) ends at position
//     pos(k) = s_1 n / r_1 + s_2 n / (r_1 r_2) + ... + s_m.
// Because the DFT matrix is symmetric, the inverse-direction transform of the
// digit-reversed data is the product of the transposed stages in reverse
// order: each stage multiplies by the conjugate twiddles first and then runs
// the conjugate butterfly on the same positions, and the result comes out in
// natural order.  Every thread writes back exactly the positions it read, so a
// stage needs one barrier and no register staging of other threads' data.
#pragma once

#include <type_traits>

#if defined(__CUDACC__)
#define ACE_HD __host__ __device__ __forceinline__
#else
#define ACE_HD inline
#endif

namespace ace {

template <typename R>
struct alignas(2 * sizeof(R)) cx {
    R re, im;
};

template <typename R>
ACE_HD cx<R> mk(R a, R b) {
    cx<R> c;
    c.re = a;
    c.im = b;
    return c;
}
template <typename R>
ACE_HD cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
ACE_HD cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
ACE_HD cx<R> cmul(cx<R> a, cx<R> b) { return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
template <typename R>
ACE_HD cx<R> scale(cx<R> a, R s) { return mk(a.re * s, a.im * s); }
// multiply by sgn * i  (sgn = +-1)
template <int SGN, typename R>
ACE_HD cx<R> mul_i(cx<R> a) { return SGN > 0 ? mk(-a.im, a.re) : mk(a.im, -a.re); }

// ------------------------------------------------------------------ codelets
// y_s = sum_q x_q w^{qs}, w = exp(SGN 2 pi i / RAD), in place on v[0..RAD).

template <int RAD, int SGN, typename R>
struct Dft;

template <int SGN, typename R>
struct Dft<2, SGN, R> {
    static ACE_HD void run(cx<R>* v) {
        cx<R> a = v[0], b = v[1];
        v[0] = a + b;
        v[1] = a - b;
    }
};

template <int SGN, typename R>
struct Dft<3, SGN, R> {
    // w = -1/2 + SGN i sqrt(3)/2
    static ACE_HD void run(cx<R>* v) {
        const R h = R(0.86602540378443864676);  // sqrt(3)/2
        cx<R> s = v[1] + v[2], d = v[1] - v[2];
        cx<R> m = v[0] - scale(s, R(0.5));
        cx<R> t = mul_i<SGN>(scale(d, h));
        v[0] = v[0] + s;
        v[1] = m + t;
        v[2] = m - t;
    }
};

template <int SGN, typename R>
struct Dft<4, SGN, R> {
    static ACE_HD void run(cx<R>* v) {
        cx<R> a = v[0] + v[2], b = v[0] - v[2];
        cx<R> c = v[1] + v[3], d = mul_i<SGN>(v[1] - v[3]);
        v[0] = a + c;
        v[2] = a - c;
        v[1] = b + d;
        v[3] = b - d;
    }
};

template <int SGN, typename R>
struct Dft<5, SGN, R> {
    // c1 = cos(2pi/5), c2 = cos(4pi/5), s1 = sin(2pi/5), s2 = sin(4pi/5)
    static ACE_HD void run(cx<R>* v) {
        const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);
        const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);
        cx<R> a1 = v[1] + v[4], b1 = v[1] - v[4];
        cx<R> a2 = v[2] + v[3], b2 = v[2] - v[3];
        cx<R> x0 = v[0];
        cx<R> p1 = x0 + scale(a1, c1) + scale(a2, c2);
        cx<R> p2 = x0 + scale(a1, c2) + scale(a2, c1);
        cx<R> q1 = mul_i<SGN>(scale(b1, s1) + scale(b2, s2));
        cx<R> q2 = mul_i<SGN>(scale(b1, s2) - scale(b2, s1));
        v[0] = x0 + a1 + a2;
        v[1] = p1 + q1;
        v[4] = p1 - q1;
        v[2] = p2 + q2;
        v[3] = p2 - q2;
    }
};

template <int SGN, typename R>
struct Dft<8, SGN, R> {
    // two radix-4 halves (even / odd inputs) joined by w8^k, k = 0..3
    static ACE_HD void run(cx<R>* v) {
        const R r = R(0.70710678118654752440);  // sqrt(2)/2
        cx<R> e[4] = {v[0], v[2], v[4], v[6]};
        cx<R> o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, SGN, R>::run(e);
        Dft<4, SGN, R>::run(o);
        // w8 = exp(SGN i pi/4) = r (1 + SGN i)
        cx<R> o1 = scale(o[1] + mul_i<SGN>(o[1]), r);
        cx<R> o2 = mul_i<SGN>(o[2]);
        cx<R> o3 = scale(mul_i<SGN>(o[3]) - o[3], r);  // w8^3 = r(-1 + SGN i)
        v[0] = e[0] + o[0];
        v[4] = e[0] - o[0];
        v[1] = e[1] + o1;
        v[5] = e[1] - o1;
        v[2] = e[2] + o2;
        v[6] = e[2] - o2;
        v[3] = e[3] + o3;
        v[7] = e[3] - o3;
    }
};

// --------------------------------------------------- compile-time twiddles
// sin and cos by their Taylor series after reduction to [-pi, pi]; evaluated
// only in constant expressions (the angles below are rational multiples of
// 2 pi known at compile time), accurate to a few ulps of double.
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double ce_reduce(double x) {
    while (x > kPi) x -= 2 * kPi;
    while (x < -kPi) x += 2 * kPi;
    return x;
}
constexpr double ce_sin(double x) {
    x = ce_reduce(x);
    double term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1));
        sum += term;
    }
    return sum;
}
constexpr double ce_cos(double x) {
    x = ce_reduce(x);
    double term = 1, sum = 1;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k - 1) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// exp(SGN 2 pi i M / N) as compile-time constants
template <int N, int M, int SGN>
struct Twiddle {
    static constexpr double re = ce_cos(2 * kPi * M / N);
    static constexpr double im = SGN * ce_sin(2 * kPi * M / N);
};

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E>
struct CLoop {
    template <class F>
    static ACE_HD void run(F&& f) {
        if constexpr (B < E) {
            f(std::integral_constant<int, B>{});
            CLoop<B + 1, E>::run(f);
        }
    }
};

// Composite codelet DFT of size A*B in registers: A-point transforms over
// the B interleaved subsequences, twiddles w_{AB}^{j s}, then B-point
// transforms; output in natural order.
template <int A, int B, int SGN, typename R>
struct DftNested {
    static ACE_HD void run(cx<R>* v) {
        cx<R> t[A * B];
        CLoop<0, B>::run([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            cx<R> u[A];
#pragma unroll
            for (int q = 0; q < A; ++q) u[q] = v[j + B * q];
            Dft<A, SGN, R>::run(u);
            CLoop<0, A>::run([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                if constexpr (j * s == 0) {
                    t[j + B * s] = u[s];
                } else {
                    const cx<R> w = mk(R(Twiddle<A * B, j * s, SGN>::re), R(Twiddle<A * B, j * s, SGN>::im));
                    t[j + B * s] = cmul(u[s], w);
                }
            });
        });
#pragma unroll
        for (int s = 0; s < A; ++s) {
            cx<R> u[B];
#pragma unroll
            for (int j = 0; j < B; ++j) u[j] = t[j + B * s];
            Dft<B, SGN, R>::run(u);
#pragma unroll
            for (int k = 0; k < B; ++k) v[s + A * k] = u[k];
        }
    }
};

template <int SGN, typename R>
struct Dft<6, SGN, R> : DftNested<2, 3, SGN, R> {};
template <int SGN, typename R>
struct Dft<9, SGN, R> : DftNested<3, 3, SGN, R> {};
template <int SGN, typename R>
struct Dft<10, SGN, R> : DftNested<2, 5, SGN, R> {};
template <int SGN, typename R>
struct Dft<12, SGN, R> : DftNested<4, 3, SGN, R> {};
template <int SGN, typename R>
struct Dft<15, SGN, R> : DftNested<5, 3, SGN, R> {};
template <int SGN, typename R>
struct Dft<16, SGN, R> : DftNested<4, 4, SGN, R> {};

// ------------------------------------------------------------------- plans

constexpr int kMaxStages = 12;

struct AxisPlan {
    int n;  // line length
    int nstages;
    int radix[kMaxStages];  // radices in forward stage order
};

// Geometry of a set of lines inside a shared-memory tile.
struct Lines {
    int n;        // length
    int nlines;   // number of lines
    int estride;  // distance between consecutive elements of a line
    int lstride;  // distance between consecutive lines
};

// Butterfly b of a stage -> (line, index within the line's butterflies).
// When a line is contiguous, consecutive b walk along it; otherwise they
// walk across lines, so a warp touches consecutive addresses either way.
ACE_HD void butterfly_coords(const Lines& L, int nb, int b, int& line, int& i) {
    if (L.estride == 1) {
        line = b / nb;
        i = b - line * nb;
    } else {
        i = b / L.nlines;
        line = b - i * L.nlines;
    }
}

// One butterfly in place: the RAD elements base[q * qstride].  tw[t] =
// exp(-2 pi i t / n); the stage's twiddles are tw[q * tstep] (tw_on = j > 0).
// SGN < 0: forward DIF (butterfly, then twiddle); SGN > 0: transposed
// conjugate stage (conjugate twiddle, then butterfly).
template <int RAD, int SGN, typename R>
ACE_HD void butterfly_core(cx<R>* base, int qstride, const cx<R>* tw, int tstep, bool tw_on) {
    cx<R> u[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) u[q] = base[q * qstride];
    if (SGN > 0 && tw_on) {
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
            cx<R> w = tw[q * tstep];
            w.im = -w.im;
            u[q] = cmul(u[q], w);
        }
    }
    Dft<RAD, SGN, R>::run(u);
    if (SGN < 0 && tw_on) {
#pragma unroll
        for (int s = 1; s < RAD; ++s) u[s] = cmul(u[s], tw[s * tstep]);
    }
#pragma unroll
    for (int s = 0; s < RAD; ++s) base[s * qstride] = u[s];
}

// Butterfly b of a stage with radix RAD on blocks of length Lb (= m RAD).
template <int RAD, int SGN, typename R>
ACE_HD void stage_butterfly(cx<R>* buf, const Lines& L, const cx<R>* tw, int Lb, int b) {
    const int m = Lb / RAD;
    const int nb = L.n / RAD;
    int line, i;
    butterfly_coords(L, nb, b, line, i);
    const int beta = i / m, j = i - beta * m;
    cx<R>* base = buf + (long long)line * L.lstride + (long long)(beta * Lb + j) * L.estride;
    butterfly_core<RAD, SGN, R>(base, m * L.estride, tw, (L.n / Lb) * j, j > 0);
}


#if defined(__CUDACC__)
template <int RAD, int SGN, typename R>
__device__ __forceinline__ void block_stage(cx<R>* buf, const Lines& L, const cx<R>* tw, int Lb) {
    const int total = (L.n / RAD) * L.nlines;
    for (int b = threadIdx.x; b < total; b += blockDim.x) stage_butterfly<RAD, SGN, R>(buf, L, tw, Lb, b);
    __syncthreads();
}

template <int SGN, typename R>
__device__ __forceinline__ void stage_dispatch(int r, cx<R>* buf, const Lines& L, const cx<R>* tw, int Lb) {
    switch (r) {
        case 2: block_stage<2, SGN, R>(buf, L, tw, Lb); break;
        case 3: block_stage<3, SGN, R>(buf, L, tw, Lb); break;
        case 4: block_stage<4, SGN, R>(buf, L, tw, Lb); break;
        case 5: block_stage<5, SGN, R>(buf, L, tw, Lb); break;
        case 6: block_stage<6, SGN, R>(buf, L, tw, Lb); break;
        case 8: block_stage<8, SGN, R>(buf, L, tw, Lb); break;
        case 9: block_stage<9, SGN, R>(buf, L, tw, Lb); break;
        case 10: block_stage<10, SGN, R>(buf, L, tw, Lb); break;
        case 12: block_stage<12, SGN, R>(buf, L, tw, Lb); break;
        case 15: block_stage<15, SGN, R>(buf, L, tw, Lb); break;
        default: block_stage<16, SGN, R>(buf, L, tw, Lb); break;
    }
}

// Full 1D transform of every line of the tile by the thread block.
// SGN < 0: natural order in, digit-reversed out.  SGN > 0: digit-reversed in,
// natural order out.
template <int SGN, typename R>
__device__ __forceinline__ void block_fft(cx<R>* buf, const Lines& L, const AxisPlan& P, const cx<R>* tw) {
    if (SGN < 0) {
        int Lb = L.n;
        for (int s = 0; s < P.nstages; ++s) {
            const int r = P.radix[s];
            stage_dispatch<SGN, R>(r, buf, L, tw, Lb);
            Lb /= r;
        }
    } else {
        int Lb = 1;
        for (int s = P.nstages - 1; s >= 0; --s) {
            const int r = P.radix[s];
            Lb *= r;
            stage_dispatch<SGN, R>(r, buf, L, tw, Lb);
        }
    }
}
#endif

// Stage radices with a register codelet.
constexpr bool is_codelet(int r) {
    return r == 2 || r == 3 || r == 4 || r == 5 || r == 6 || r == 8 || r == 9 || r == 10 || r == 12 || r == 15 ||
           r == 16;
}

// Factor n into as few codelet radices as possible, preferring the largest
// smallest radix (balanced stages); the larger radix goes first.  Returns
// false when n has a prime factor above 5 or needs more than kMaxStages.
constexpr bool make_axis_plan(int n, AxisPlan& P) {
    P.n = n;
    P.nstages = 0;
    if (n < 1) return false;
    if (n == 1) return true;
    if (is_codelet(n)) {
        P.radix[P.nstages++] = n;
        return true;
    }
    int best1 = 0, best2 = 0;
    for (int r1 = 16; r1 >= 2; --r1)
        if (is_codelet(r1) && n % r1 == 0 && is_codelet(n / r1)) {
            const int r2 = n / r1, lo = r1 < r2 ? r1 : r2;
            const int blo = best1 < best2 ? best1 : best2;
            if (best1 == 0 || lo > blo || (lo == blo && r1 > best1)) {
                best1 = r1;
                best2 = r2;
            }
        }
    if (best1) {
        P.radix[P.nstages++] = best1;
        P.radix[P.nstages++] = best2;
        return true;
    }
    int m = n;
    const int order[11] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
    while (m > 1) {
        int pick = 0;
        for (int r : order)
            if (m % r == 0) {
                pick = r;
                break;
            }
        if (pick == 0 || P.nstages == kMaxStages) return false;
        P.radix[P.nstages++] = pick;
        m /= pick;
    }
    return true;
}

// Two stages with the given first radix: r0, then n / r0 (both codelets).
// The candidates the plan autotuner times for one axis length.
constexpr bool make_axis_plan_first(int n, int r0, AxisPlan& P) {
    P.n = n;
    P.nstages = 0;
    if (r0 < 2 || n % r0 != 0 || !is_codelet(r0) || !is_codelet(n / r0)) return false;
    P.radix[P.nstages++] = r0;
    P.radix[P.nstages++] = n / r0;
    return true;
}

// Compile-time plan of an axis of length N: make_axis_plan's choice (R0 = 0)
// or the two stages R0, N / R0.
template <int N, int R0 = 0>
struct CPlan {
    static constexpr AxisPlan P = [] {
        AxisPlan p{};
        if (R0 == 0)
            make_axis_plan(N, p);
        else
            make_axis_plan_first(N, R0, p);
        return p;
    }();
    static_assert(R0 == 0 || P.nstages == 2, "R0 and N / R0 must both be codelet radices");
    static constexpr int stages = P.nstages;
    static constexpr int radix(int s) { return P.radix[s]; }
    static constexpr int block_len(int s) {
        int L = N;
        for (int t = 0; t < s; ++t) L /= P.radix[t];
        return L;
    }
};

#if defined(__CUDACC__)
// The same stages with every size known at compile time (N, line count and
// strides, thread count NT): index arithmetic folds to shifts and multiplies.
template <int RAD, int SGN, int N, int LB, int NLINES, int ESTRIDE, int LSTRIDE, int NT, typename R>
__device__ __forceinline__ void static_stage(cx<R>* buf, const cx<R>* tw) {
    constexpr int M = LB / RAD, NB = N / RAD, TOTAL = NB * NLINES, TS = N / LB;
    if constexpr (ESTRIDE == 1 && M > 1 && NT % NB == 0) {
        // contiguous lines, NT a multiple of the butterflies per line: every
        // butterfly of this thread has the same j, so its twiddles are read once
        const int i = (int)threadIdx.x % NB, beta = i / M, j = i - beta * M;
        cx<R> w[RAD];
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
            w[q] = tw[q * TS * j];
            if (SGN > 0) w[q].im = -w[q].im;
        }
        const bool tw_on = j > 0;
#pragma unroll 2
        for (int line = (int)threadIdx.x / NB; line < NLINES; line += NT / NB) {
            cx<R>* base = buf + line * LSTRIDE + beta * LB + j;
            cx<R> u[RAD];
#pragma unroll
            for (int q = 0; q < RAD; ++q) u[q] = base[q * M];
            if (SGN > 0 && tw_on) {
#pragma unroll
                for (int q = 1; q < RAD; ++q) u[q] = cmul(u[q], w[q]);
            }
            Dft<RAD, SGN, R>::run(u);
            if (SGN < 0 && tw_on) {
#pragma unroll
                for (int q = 1; q < RAD; ++q) u[q] = cmul(u[q], w[q]);
            }
#pragma unroll
            for (int q = 0; q < RAD; ++q) base[q * M] = u[q];
        }
        __syncthreads();
        return;
    }
#pragma unroll 2
    for (int b = threadIdx.x; b < TOTAL; b += NT) {
        int line, i;
        if constexpr (ESTRIDE == 1) {
            line = b / NB;
            i = b - line * NB;
        } else {
            i = b / NLINES;
            line = b - i * NLINES;
        }
        const int beta = i / M, j = i - beta * M;
        butterfly_core<RAD, SGN, R>(buf + line * LSTRIDE + (beta * LB + j) * ESTRIDE, M * ESTRIDE, tw, TS * j,
                                    M > 1 && j > 0);
    }
    __syncthreads();
}

template <int SGN, int N, int NLINES, int ESTRIDE, int LSTRIDE, int NT, typename R, int R0 = 0>
__device__ __forceinline__ void static_fft(cx<R>* buf, const cx<R>* tw) {
    using PL = CPlan<N, R0>;
    CLoop<0, PL::stages>::run([&](auto sc) {
        constexpr int s = SGN < 0 ? decltype(sc)::value : PL::stages - 1 - decltype(sc)::value;
        static_stage<PL::radix(s), SGN, N, PL::block_len(s), NLINES, ESTRIDE, LSTRIDE, NT, R>(buf, tw);
    });
}
#endif

// Position of frequency k after the forward transform (see the header note).
constexpr int digit_reversed_position(const AxisPlan& P, int k) {
    int pos = 0, span = P.n;
    for (int s = 0; s < P.nstages; ++s) {
        const int r = P.radix[s];
        span /= r;
        pos += (k % r) * span;
        k /= r;
    }
    return pos;
}

}  // namespace ace
