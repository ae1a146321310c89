// cube_dispatch.cu -- route a pass to the compile-time kernel of its N^3 box.
#include "pass_kernel.cuh"
#include "pipeline.cuh"
#include "plane.cuh"
#include "zline.cuh"
#include "halfplane.cuh"

namespace ace {

namespace pass_detail {
#define ACE_CUBE_DECL(N)                                                                                      \
    extern template cudaError_t dispatch_cube<N>(const PassArgs&, const PassShape&, int, int, int, int, int, \
                                                 cudaStream_t);
ACE_CUBE_DECL(32)
ACE_CUBE_DECL(60)
ACE_CUBE_DECL(80)
ACE_CUBE_DECL(90)
ACE_CUBE_DECL(96)
ACE_CUBE_DECL(100)
ACE_CUBE_DECL(108)
ACE_CUBE_DECL(120)
ACE_CUBE_DECL(160)
#undef ACE_CUBE_DECL
}  // namespace pass_detail

// the pair passes' alternative radix plans (pair_radix_alternatives), in cube_r*.cu
#define ACE_ALT_PLANS(X) X(96, 8) X(96, 16) X(120, 10) X(120, 8) X(160, 10)
#define ACE_ALT_PIPE_PLANS(X) X(96, 8) X(96, 16) X(160, 10)
namespace pass_detail {
#define ACE_ALT_CUBE_DECL(N, F)                                                                                  \
    extern template cudaError_t dispatch_cube<N, F>(const PassArgs&, const PassShape&, int, int, int, int, int, \
                                                    cudaStream_t);
ACE_ALT_PLANS(ACE_ALT_CUBE_DECL)
#undef ACE_ALT_CUBE_DECL
}  // namespace pass_detail
#define ACE_ALT_DECL(N, F)                                                              \
    extern template cudaError_t zline_launch<N, F>(const PassArgs&, int, cudaStream_t); \
    extern template cudaError_t tplane_launch<N, F>(int, const PassArgs&, int, cudaStream_t);
ACE_ALT_PLANS(ACE_ALT_DECL)
#undef ACE_ALT_DECL
#define ACE_ALT_PIPE_DECL(N, F) \
    extern template cudaError_t pipeline_launch<N, F>(const PassArgs&, const PipeArgs&, cudaStream_t);
ACE_ALT_PIPE_PLANS(ACE_ALT_PIPE_DECL)
#undef ACE_ALT_PIPE_DECL

// (n, first radix) as one switch key
constexpr int alt_key(int n, int r0) { return n * 32 + r0; }

#define ACE_ZLINE_DECL(N) extern template cudaError_t zline_launch<N>(const PassArgs&, int, cudaStream_t);
ACE_ZLINE_DECL(32)
ACE_ZLINE_DECL(60)
ACE_ZLINE_DECL(80)
ACE_ZLINE_DECL(90)
ACE_ZLINE_DECL(96)
ACE_ZLINE_DECL(100)
ACE_ZLINE_DECL(108)
ACE_ZLINE_DECL(120)
ACE_ZLINE_DECL(160)
#undef ACE_ZLINE_DECL

cudaError_t zline_coulomb_launch(int n, const PassArgs& a, int batch, cudaStream_t st) {
    if (a.r0 != 0) {
        switch (alt_key(n, a.r0)) {
#define ACE_ALT_CASE(N, F) \
    case alt_key(N, F): return zline_launch<N, F>(a, batch, st);
            ACE_ALT_PLANS(ACE_ALT_CASE)
#undef ACE_ALT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    switch (n) {
        case 32: return zline_launch<32>(a, batch, st);
        case 60: return zline_launch<60>(a, batch, st);
        case 80: return zline_launch<80>(a, batch, st);
        case 90: return zline_launch<90>(a, batch, st);
        case 96: return zline_launch<96>(a, batch, st);
        case 100: return zline_launch<100>(a, batch, st);
        case 108: return zline_launch<108>(a, batch, st);
        case 120: return zline_launch<120>(a, batch, st);
        case 160: return zline_launch<160>(a, batch, st);
        default: return cudaErrorInvalidValue;
    }
}

#define ACE_TPLANE_DECL(N) extern template cudaError_t tplane_launch<N>(int, const PassArgs&, int, cudaStream_t);
ACE_TPLANE_DECL(32)
ACE_TPLANE_DECL(60)
ACE_TPLANE_DECL(80)
ACE_TPLANE_DECL(90)
ACE_TPLANE_DECL(96)
ACE_TPLANE_DECL(100)
ACE_TPLANE_DECL(108)
ACE_TPLANE_DECL(120)
ACE_TPLANE_DECL(160)
#undef ACE_TPLANE_DECL

cudaError_t tplane_pair_launch(int n, int which, const PassArgs& a, int batch, cudaStream_t st) {
    if (a.r0 != 0) {
        switch (alt_key(n, a.r0)) {
#define ACE_ALT_CASE(N, F) \
    case alt_key(N, F): return tplane_launch<N, F>(which, a, batch, st);
            ACE_ALT_PLANS(ACE_ALT_CASE)
#undef ACE_ALT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    switch (n) {
        case 32: return tplane_launch<32>(which, a, batch, st);
        case 60: return tplane_launch<60>(which, a, batch, st);
        case 80: return tplane_launch<80>(which, a, batch, st);
        case 90: return tplane_launch<90>(which, a, batch, st);
        case 96: return tplane_launch<96>(which, a, batch, st);
        case 100: return tplane_launch<100>(which, a, batch, st);
        case 108: return tplane_launch<108>(which, a, batch, st);
        case 120: return tplane_launch<120>(which, a, batch, st);
        case 160: return tplane_launch<160>(which, a, batch, st);
        default: return cudaErrorInvalidValue;
    }
}

#define ACE_PIPE_DECL(N) extern template cudaError_t pipeline_launch<N>(const PassArgs&, const PipeArgs&, cudaStream_t);
ACE_PIPE_DECL(32)
ACE_PIPE_DECL(80)
ACE_PIPE_DECL(96)
ACE_PIPE_DECL(160)
#undef ACE_PIPE_DECL

cudaError_t pipeline_pair_launch(int n, const PassArgs& a, const PipeArgs& p, cudaStream_t st) {
    if (a.r0 != 0) {
        switch (alt_key(n, a.r0)) {
#define ACE_ALT_CASE(N, F) \
    case alt_key(N, F): return pipeline_launch<N, F>(a, p, st);
            ACE_ALT_PIPE_PLANS(ACE_ALT_CASE)
#undef ACE_ALT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    switch (n) {
        case 32: return pipeline_launch<32>(a, p, st);
        case 80: return pipeline_launch<80>(a, p, st);
        case 96: return pipeline_launch<96>(a, p, st);
        case 160: return pipeline_launch<160>(a, p, st);
        default: return cudaErrorInvalidValue;
    }
}

extern template cudaError_t halfplane_launch<120>(int, const PassArgs&, int, cudaStream_t);
extern template cudaError_t halfplane_launch<120, 10>(int, const PassArgs&, int, cudaStream_t);
extern template cudaError_t halfplane_launch<120, 8>(int, const PassArgs&, int, cudaStream_t);

cudaError_t halfplane_pair_launch(int n, int which, const PassArgs& a, int batch, cudaStream_t st) {
    switch (alt_key(n, a.r0)) {
        case alt_key(120, 0): return halfplane_launch<120>(which, a, batch, st);
        case alt_key(120, 10): return halfplane_launch<120, 10>(which, a, batch, st);
        case alt_key(120, 8): return halfplane_launch<120, 8>(which, a, batch, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t cube_pass_launch(int n, const PassArgs& a, const PassShape& s, int pro, int epi, int mid, int sgn,
                             int batch, cudaStream_t st) {
    using namespace pass_detail;
    if (a.r0 != 0) {
        switch (alt_key(n, a.r0)) {
#define ACE_ALT_CASE(N, F) \
    case alt_key(N, F): return dispatch_cube<N, F>(a, s, pro, epi, mid, sgn, batch, st);
            ACE_ALT_PLANS(ACE_ALT_CASE)
#undef ACE_ALT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    switch (n) {
        case 32: return dispatch_cube<32>(a, s, pro, epi, mid, sgn, batch, st);
        case 60: return dispatch_cube<60>(a, s, pro, epi, mid, sgn, batch, st);
        case 80: return dispatch_cube<80>(a, s, pro, epi, mid, sgn, batch, st);
        case 90: return dispatch_cube<90>(a, s, pro, epi, mid, sgn, batch, st);
        case 96: return dispatch_cube<96>(a, s, pro, epi, mid, sgn, batch, st);
        case 100: return dispatch_cube<100>(a, s, pro, epi, mid, sgn, batch, st);
        case 108: return dispatch_cube<108>(a, s, pro, epi, mid, sgn, batch, st);
        case 120: return dispatch_cube<120>(a, s, pro, epi, mid, sgn, batch, st);
        case 160: return dispatch_cube<160>(a, s, pro, epi, mid, sgn, batch, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ace
