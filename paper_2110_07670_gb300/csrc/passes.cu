// passes.cu -- the FFT pass kernel of the pair Poisson solves.
//
// A 3D transform of an n0 x n1 x n2 box is done in passes; each thread block
// owns one tile of one transform in shared memory, transforms it along one or
// more axes with the in-place stages of fft_core.cuh, and hands it to an
// epilogue.  The prologues and epilogues fuse the exchange work of
// arXiv:2110.07670 Section 2.1 into the first and last passes:
//
//   pair density (Eq. 3)       rho = f_a phi_b, two pairs packed as re + i im
//   Coulomb solve (Eq. 3)      v(G) = 4 pi / |G|^2 rho(G) / N, G = 0 dropped,
//                              applied between the forward and inverse z axis
//   exchange (Eq. 2)           W_a += v phi_b, W_b += v f_a (a != b)
//   pair energy (Eq. 4)        e_ab = sum_r rho v  (times Omega / N later)
//
// so pair densities and pair potentials never travel through global memory
// between the passes; only the half-transformed spectrum does.
#include <cstdio>

#include "internal.h"

namespace ace {

namespace {

__device__ __forceinline__ int fold_index(int i, int n) { return i < n - n / 2 ? i : i - n; }

template <typename R>
__device__ __forceinline__ void atomic_add_real(R* p, R v) {
    atomicAdd(p, v);
}

template <typename R, int PRO, int EPI, int MID, int SGN>
__global__ void __launch_bounds__(512) tile_pass(PassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile_elems = a.tz * a.ty * a.tx;
    cx<R>* tile = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* twx = tile + tile_elems;
    cx<R>* twy = twx + ((a.axes & 1) ? a.n2 : 0);
    cx<R>* twz = twy + ((a.axes & 2) ? a.n1 : 0);
    int* fq = reinterpret_cast<int*>(twz + ((a.axes & 4) ? a.n0 : 0));  // frequency of each position (Coulomb)
    if (MID == MID_COULOMB) {
        for (int j = threadIdx.x; j < a.n0; j += blockDim.x) fq[j] = a.freq[0][j];
        for (int j = threadIdx.x; j < a.n1; j += blockDim.x) fq[a.n0 + j] = a.freq[1][j];
        for (int j = threadIdx.x; j < a.n2; j += blockDim.x) fq[a.n0 + a.n1 + j] = a.freq[2][j];
    }
    if (a.axes & 1)
        for (int j = threadIdx.x; j < a.n2; j += blockDim.x) twx[j] = reinterpret_cast<const cx<R>*>(a.twx)[j];
    if (a.axes & 2)
        for (int j = threadIdx.x; j < a.n1; j += blockDim.x) twy[j] = reinterpret_cast<const cx<R>*>(a.twy)[j];
    if (a.axes & 4)
        for (int j = threadIdx.x; j < a.n0; j += blockDim.x) twz[j] = reinterpret_cast<const cx<R>*>(a.twz)[j];

    const int t = blockIdx.y;
    const int tiles_x = a.n2 / a.tx, tiles_y = a.n1 / a.ty;
    const int tile_id = blockIdx.x;
    const int bx = tile_id % tiles_x, by = (tile_id / tiles_x) % tiles_y, bz = tile_id / (tiles_x * tiles_y);
    const int z0 = bz * a.tz, y0 = by * a.ty, x0 = bx * a.tx;
    const long long N = (long long)a.n0 * a.n1 * a.n2;
    const int txy = a.tx * a.ty;

    Quad q = {0, 0, -1, 0};
    if (PRO != PRO_LOAD || EPI != EPI_STORE) q = a.quads[a.t0 + t];
    const R* fl = reinterpret_cast<const R*>(a.fl);
    const R* fr = reinterpret_cast<const R*>(a.fr);

    // ---- prologue: global -> tile
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        const int ex = e % a.tx, ey = (e / a.tx) % a.ty, ez = e / txy;
        const long long r = ((long long)(z0 + ez) * a.n1 + (y0 + ey)) * a.n2 + (x0 + ex);
        cx<R> v;
        if (PRO == PRO_LOAD) {
            v = reinterpret_cast<const cx<R>*>(a.src)[(long long)t * a.src_tstride + r];
        } else if (PRO == PRO_PAIR) {
            v.re = fl[q.a * N + r] * fr[q.b * N + r];
            v.im = q.c >= 0 ? fl[q.c * N + r] * fr[q.d * N + r] : R(0);
        } else {
            v.re = fl[q.a * N + r];
            v.im = q.c >= 0 ? fl[q.c * N + r] : R(0);
        }
        tile[e] = v;
    }
    __syncthreads();

    // ---- transforms
    if (a.axes & 1) {
        Lines L = {a.tx, a.tz * a.ty, 1, a.tx};
        block_fft<SGN, R>(tile, L, a.px, twx);
    }
    if (a.axes & 2) {
        Lines L = {a.ty, a.tx, a.tx, 1};
        block_fft<SGN, R>(tile, L, a.py, twy);
    }
    if (a.axes & 4) {
        Lines L = {a.tz, txy, txy, 1};
        if (MID == MID_COULOMB) {
            block_fft<-1, R>(tile, L, a.pz, twz);
            const R four_pi_s = R(4.0 * 3.14159265358979323846 * a.kscale);
            for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
                const int ex = e % a.tx, ey = (e / a.tx) % a.ty, ez = e / txy;
                // positions hold digit-reversed frequencies after the forward stages
                const R h = R(fold_index(fq[z0 + ez], a.n0)), k = R(fold_index(fq[a.n0 + y0 + ey], a.n1)),
                        l = R(fold_index(fq[a.n0 + a.n1 + x0 + ex], a.n2));
                const R gx = h * R(a.b[0]) + k * R(a.b[3]) + l * R(a.b[6]);
                const R gy = h * R(a.b[1]) + k * R(a.b[4]) + l * R(a.b[7]);
                const R gz = h * R(a.b[2]) + k * R(a.b[5]) + l * R(a.b[8]);
                const R g2 = gx * gx + gy * gy + gz * gz;
                const R kv = g2 > R(0) ? four_pi_s / g2 : R(0);
                tile[e] = scale(tile[e], kv);
            }
            __syncthreads();
            block_fft<+1, R>(tile, L, a.pz, twz);
        } else {
            block_fft<SGN, R>(tile, L, a.pz, twz);
        }
    }

    // ---- epilogue: tile -> global
    R e1 = R(0), e2 = R(0);
    R* accl = reinterpret_cast<R*>(a.accl);
    R* accr = reinterpret_cast<R*>(a.accr);
    for (int e = threadIdx.x; e < tile_elems; e += blockDim.x) {
        const int ex = e % a.tx, ey = (e / a.tx) % a.ty, ez = e / txy;
        const long long r = ((long long)(z0 + ez) * a.n1 + (y0 + ey)) * a.n2 + (x0 + ex);
        const cx<R> v = tile[e];
        if (EPI == EPI_STORE) {
            reinterpret_cast<cx<R>*>(a.dst)[(long long)t * a.dst_tstride + r] = v;
        } else if (EPI == EPI_SPLIT) {
            accl[q.a * N + r] = v.re * R(a.scale);
            if (q.c >= 0) accl[q.c * N + r] = v.im * R(a.scale);
        } else {
            const R la = fl[q.a * N + r], rb = fr[q.b * N + r];
            e1 += la * rb * v.re;
            atomic_add_real(accl + q.a * N + r, v.re * rb);
            if (a.symmetric && q.a != q.b) atomic_add_real(accr + q.b * N + r, v.re * la);
            if (q.c >= 0) {
                const R lc = fl[q.c * N + r], rd = fr[q.d * N + r];
                e2 += lc * rd * v.im;
                atomic_add_real(accl + q.c * N + r, v.im * rd);
                if (a.symmetric && q.c != q.d) atomic_add_real(accr + q.d * N + r, v.im * lc);
            }
        }
    }
    if (EPI == EPI_ACCUM && a.e_part != nullptr) {
        double d1 = double(e1), d2 = double(e2);
        for (int o = 16; o > 0; o >>= 1) {
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        __syncthreads();  // tile no longer needed; reuse it for the reduction
        double* red = reinterpret_cast<double*>(smem_raw);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        if (lane == 0) {
            red[2 * warp] = d1;
            red[2 * warp + 1] = d2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s1 = 0, s2 = 0;
            for (int w = 0; w < nw; ++w) {
                s1 += red[2 * w];
                s2 += red[2 * w + 1];
            }
            const long long ntiles = gridDim.x;
            double* dst = a.e_part + ((long long)(a.t0 + t) * ntiles + tile_id) * 2;
            dst[0] = s1;
            dst[1] = s2;
        }
    }
}

template <typename R, int PRO, int EPI, int MID, int SGN>
cudaError_t launch_one(const PassArgs& a, const PassShape& s, int batch, cudaStream_t st) {
    auto k = tile_pass<R, PRO, EPI, MID, SGN>;
    if (s.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
        if (e != cudaSuccess) return e;
    }
    const int ntiles = (a.n0 / s.tz) * (a.n1 / s.ty) * (a.n2 / s.tx);
    dim3 grid(ntiles, batch);
    k<<<grid, s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace


template <typename R>
cudaError_t launch_pass(const PassArgs& a0, const PassShape& s, int pro, int epi, int mid, int sgn, int batch,
                        cudaStream_t st) {
    PassArgs a = a0;
    a.tz = s.tz;
    a.ty = s.ty;
    a.tx = s.tx;
    a.axes = s.axes;
    if (batch <= 0) return cudaSuccess;
    if (mid == MID_COULOMB) return launch_one<R, PRO_LOAD, EPI_STORE, MID_COULOMB, -1>(a, s, batch, st);
    if (pro == PRO_LOAD && epi == EPI_STORE)
        return sgn < 0 ? launch_one<R, PRO_LOAD, EPI_STORE, MID_NONE, -1>(a, s, batch, st)
                       : launch_one<R, PRO_LOAD, EPI_STORE, MID_NONE, +1>(a, s, batch, st);
    if (pro == PRO_PAIR && epi == EPI_STORE && sgn < 0)
        return launch_one<R, PRO_PAIR, EPI_STORE, MID_NONE, -1>(a, s, batch, st);
    if (pro == PRO_LOAD && epi == EPI_ACCUM && sgn > 0)
        return launch_one<R, PRO_LOAD, EPI_ACCUM, MID_NONE, +1>(a, s, batch, st);
    if (pro == PRO_LOAD && epi == EPI_SPLIT && sgn > 0)
        return launch_one<R, PRO_LOAD, EPI_SPLIT, MID_NONE, +1>(a, s, batch, st);
    if (pro == PRO_PACK2 && epi == EPI_STORE && sgn < 0)
        return launch_one<R, PRO_PACK2, EPI_STORE, MID_NONE, -1>(a, s, batch, st);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_pass<float>(const PassArgs&, const PassShape&, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_pass<double>(const PassArgs&, const PassShape&, int, int, int, int, int, cudaStream_t);

}  // namespace ace
