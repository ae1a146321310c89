// noalloc.cu -- ace_apply_noalloc: the ACE apply for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they apply the
// operator: an inner loop that must not stall (cudaMalloc and cudaFree
// synchronise the whole device), or a host whose device memory is owned by
// another allocator or fixed at start-up.  This entry point needs no plan and
// allocates nothing: its working memory is one file-scope __device__ array,
// loaded with the library and held on every device that uses it until the
// process exits.
#include <algorithm>
#include <mutex>
#include <string>

#include "ace.h"
#include "internal.h"

namespace {

constexpr long long kScratchDoubles = 1LL << 20;  // 8 MiB of doubles per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_apply_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_apply_scratch on the current device, looked up once per
// device.  In host code the array's name only stands in for it; the address
// must come from cudaGetSymbolAddress with that device current.
int scratch_on_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return ace::set_last_error(ACE_ERR_CUDA, "ace_apply_noalloc: no usable current device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
        if (e != cudaSuccess || p == nullptr)
            return ace::set_last_error(
                ACE_ERR_CUDA, (std::string("ace_apply_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)).c_str());
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ACE_OK;
}

template <typename R>
int apply_noalloc(const void* xi, int n_occ, const void* psi, int T, int npw, void* Kpsi, cudaStream_t st) {
    const long long K = 2LL * npw;
    const long long mn = (long long)T * n_occ;
    // C[t][k] needs T n_occ doubles and each Gram partial another T n_occ
    if (2 * mn > kScratchDoubles) {
        const std::string msg = "ace_apply_noalloc: T * n_occ = " + std::to_string(mn) + " exceeds the limit of " +
                                std::to_string(kScratchDoubles / 2) + " (8 MiB of device scratch)";
        return ace::set_last_error(ACE_ERR_INVALID_ARG, msg.c_str());
    }
    double* scratch = nullptr;
    const int s = scratch_on_current_device(&scratch);
    if (s != ACE_OK) return s;
    const int tiles = ((T + 63) / 64) * ((n_occ + 63) / 64);
    long long nchunk = std::max(1, (2 * 152 + tiles - 1) / tiles);
    nchunk = std::min<long long>(nchunk, std::max<long long>(1, K / 256));
    nchunk = std::min<long long>(nchunk, kScratchDoubles / mn - 1);
    double* C = scratch;
    double* part = scratch + mn;
    const R* x = static_cast<const R*>(xi);
    const R* p = static_cast<const R*>(psi);
    cudaError_t e = ace::launch_gram_partial<R>(p, x, T, n_occ, K, (int)nchunk, part, st);
    if (e == cudaSuccess) e = ace::launch_gram_finish<R>(part, (int)nchunk, p, x, T, n_occ, K, C, n_occ, st);
    if (e == cudaSuccess) e = ace::launch_gemm_nn<R>(C, T, n_occ, x, K, -1.0, static_cast<R*>(Kpsi), false, st);
    if (e != cudaSuccess)
        return ace::set_last_error(ACE_ERR_CUDA, (std::string("ace_apply_noalloc: ") + cudaGetErrorString(e)).c_str());
    return ACE_OK;
}

}  // namespace

extern "C" int ace_apply_noalloc(const void* xi, int n_occ, const void* psi, int T, int n_pw_half, int precision,
                                 void* Kpsi, void* stream) {
    if (!xi || (T > 0 && (!psi || !Kpsi)))
        return ace::set_last_error(ACE_ERR_INVALID_ARG, "ace_apply_noalloc: null argument");
    if (n_occ < 1 || T < 0 || n_pw_half < 1 || (precision != ACE_FP64 && precision != ACE_MIXED))
        return ace::set_last_error(ACE_ERR_INVALID_ARG,
                                   "ace_apply_noalloc: need n_occ >= 1, T >= 0, n_pw_half >= 1, ACE_FP64 or ACE_MIXED");
    if (T == 0) return ACE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return precision == ACE_FP64 ? apply_noalloc<double>(xi, n_occ, psi, T, n_pw_half, Kpsi, st)
                                 : apply_noalloc<float>(xi, n_occ, psi, T, n_pw_half, Kpsi, st);
}
