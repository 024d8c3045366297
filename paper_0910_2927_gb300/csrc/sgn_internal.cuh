// Internal declarations shared by the CUDA translation units of libsgn.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sgn.h"

namespace sgn {

// ----------------------------------------------------------------- errors --
void set_error(const std::string& msg);
#define SGN_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess) {                                                       \
            ::sgn::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));      \
            return SGN_ERR_CUDA;                                                       \
        }                                                                              \
    } while (0)
#define SGN_CHECK(call)            \
    do {                           \
        int _s = (call);           \
        if (_s != SGN_OK) return _s; \
    } while (0)

// Kernel launches issued by this host thread (launch helpers add 1 each; a graph
// replay adds its kernel-node count).
extern thread_local long long g_launches;
inline void count_launch(long long k = 1) { g_launches += k; }

// ---------------------------------------------------------------- complex --
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Exact division of n < 2^27 by a fixed d >= 1 with one 64-bit multiply and a
// shift: M = floor(2^(32+s) / d) + 1, 2^s >= d.  The error n (M - 2^(32+s)/d) /
// 2^(32+s) < 2^27 / 2^(32+s) <= 1/(32 d) never crosses an integer.
struct FastDiv {
    uint32_t d = 1;
    int sh = 32;
    uint64_t M = (uint64_t(1) << 32) + 1;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div) {
        int s = 0;
        while ((1u << s) < div) ++s;
        sh = 32 + s;
        M = (uint64_t(1) << sh) / div + 1;
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((uint64_t)n * M) >> sh); }
};

// Lattice geometry and operator parameters passed by value to the stencil.
struct StencilParams {
    int L[4];          // Lx, Ly, Lz, Lt
    int64_t vol;       // sites
    int64_t stride_rhs;  // complex elements between consecutive fields (= 12 vol)
    double diag;       // 4 + m_W
    double cf[4];      // forward hop coefficient -1/2 e^{+mu d_nu,t}
    double cb[4];      // backward hop coefficient -1/2 e^{-mu d_nu,t}
    int ap[4];         // antiperiodic flags
    // the same coefficients in FP32 for the FP32 stencil (no FP64 conversion in the kernel)
    float diag32;
    float cf32[4];
    float cb32[4];
    // the FP32 roundings of the remainders (diag - diag32 etc.): the float-float stencil's constants
    float diag_lo;
    float cf_lo[4];
    float cb_lo[4];
    FastDiv div[3];    // by Lx, Ly, Lz (site < 2^27)
};

// ---------------------------------------------------------- field layout --
// Inside the library every field is kept "packed": the complex entry k = 3 spin
// + colour of site s of a field of vol sites sits at (k/2) * 2 vol + 2 s + k%2,
// i.e. six planes that each hold two consecutive spin-colour entries per site.
// A warp of 32 consecutive sites then reads 32 x 16 contiguous bytes per plane
// (FP32), where the natural [site][12] order reads every 96th-byte chunk.
// Links are packed as [dir][row 3][col 3][site].  Dot products and vector
// updates do not depend on the order; only the stencil and the boundary do.
template <class T>
cudaError_t pack_fields(const T* natural, T* packed, int64_t vol, int nfield, cudaStream_t st);
template <class T>
cudaError_t unpack_fields(const T* packed, T* natural, int64_t vol, int nfield, cudaStream_t st);
cudaError_t pack_links(const double2* natural, double2* packed, int64_t vol, cudaStream_t st);

// ---------------------------------------------------------- kernel entry --
// Stencil: out = H_W in for nrhs fields (packed layout).  Real = double or float; links in
// double, float or bf16 (Link).  skip: per-field flags (non-zero: skip), may be null.
// Launch shape: sx sites (x fastest) by rb threads per CTA, each thread nr
// fields of its site (nr <= 3 FP32, 1 FP64); {0, 0, 1} picks the default.
// pipe = 1 selects the FP32 kernel that stages neighbour spinors through shared
// memory with cp.async (a stage ahead of the computation; nr <= 2); pipe = 2 the
// FP32 kernel with paired (FFMA2) arithmetic over two fields (nr = 2), pipe = 3 the
// same kernel capped at 128 registers.
struct StencilShape {
    int sx = 0;
    int rb = 0;
    int nr = 1;
    int pipe = 0;
};
cudaError_t launch_hw_f64(double2* out, const double2* in, const double2* U, int nrhs,
                          const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh = {});
cudaError_t launch_hw_f32(float2* out, const float2* in, const float2* U, int nrhs,
                          const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh = {});
cudaError_t launch_hw_f32_bf16links(float2* out, const float2* in, const __nv_bfloat162* U, int nrhs,
                                    const StencilParams& p, const int* skip, cudaStream_t st,
                                    StencilShape sh = {});
cudaError_t launch_hw_f32_f16links(float2* out, const float2* in, const __half2* U, int nrhs,
                                   const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh = {});
// Float-float stencil (stencil_ff.cu): fields as (hi, lo) pairs of packed FP32 fields, links as
// one float4 (U32, fl(U - U32)) per packed entry; about 1e-13 of the FP64 result.
cudaError_t launch_hw_ff(float2* oh, float2* ol, const float2* ih, const float2* il, const float4* Uf, int nrhs,
                         const StencilParams& p, cudaStream_t st);
// FP64 <-> (hi, lo) conversions of count complex entries, the FP64 true residual
// r = b - (yh + yl) + sigma x, and the float-float links (U32, fl(U - U32)).
cudaError_t split_ff(const double2* in, float2* hi, float2* lo, int64_t count, cudaStream_t st);
cudaError_t join_ff(const float2* hi, const float2* lo, double2* out, int64_t count, cudaStream_t st);
cudaError_t residual_ff(double2* r, const double2* b, const float2* yh, const float2* yl, double sigma,
                        const double2* x, int64_t count, cudaStream_t st);
cudaError_t links_ff(const double2* U, const float2* U32, float4* out, int64_t count, cudaStream_t st);

// ------------------------------------------------------------ vector ops --
// A "basis" is J fields per column: element e of vector j of column r lives at
// base[j * sj + r * sr + e] (sr = 0 for a basis shared by every column).
template <class T>
struct Basis {
    const T* base;
    int64_t sj;
    int64_t sr;
};

// Block layout of the two-stage reductions: partials[(r * stride + j) * nblk + b].
struct Reduce {
    double2* partial;  // scratch
    int nblk;          // blocks per column
    int stride;        // slots per column (>= J + 1)
};

}  // namespace sgn
