// Tall-skinny products with a small basis V (J <= 64 fields) against many
// columns W (one field each): the deflation projection of the mixed form's
// refinement, L^dag r_i and r_i -= R c_i, x_i += R d_i for every shifted system
// (Sec. 4, eqs. (4.2)-(4.5), applied to the s * nrhs true residuals).  The
// column-by-column kernels of blas.cu re-read V for every column (240 columns x
// 30 fields); here a CTA stages a row chunk of V in shared memory once and uses
// it for a tile of columns, so V comes from HBM once and from L2 once per tile.
//
// Arithmetic: products and the sum over a CTA's rows in FP32 (V in its FP32
// copy, W converted on load), the sum over CTAs in FP64.  The results are
// corrections of size ~1e-6 ||b~|| in refinement, where an FP32 relative error
// is far below every tolerance; the FP64 form does not use these kernels.
#include "blas.cuh"

namespace sgn {
namespace {

constexpr int TN_THREADS = 256;
constexpr int TN_TR = 32;  // rows per shared-memory chunk
constexpr int TN_NC = 16;  // columns per CTA
constexpr int TN_JMAX = 64;

__device__ __forceinline__ float2 ld_f2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_f2(const double2* p) {
    const double2 v = __ldg(p);
    return make_float2((float)v.x, (float)v.y);
}

// partial[((col * rstride + j) * nblk + b)] = sum over this CTA's rows of conj(V_j) W_col,
// the layout the second-stage reduction (k_reduce, RM_STORE) sums over b.
template <class TV>
__global__ void __launch_bounds__(TN_THREADS)
    k_tsmm_tn(const TV* __restrict__ V, int64_t sv, int J, const double2* __restrict__ W, int64_t sw, int N,
              int64_t n, int64_t rows_per_cta, double2* __restrict__ partial, int rstride, int nblk) {
    __shared__ float2 Vs[TN_JMAX][TN_TR];
    __shared__ float2 Ws[TN_NC][TN_TR + 1];  // padded: lanes of different columns hit different banks
    const int t = threadIdx.x;
    const int b = blockIdx.x;
    const int c0 = blockIdx.y * TN_NC;
    const int64_t r0 = (int64_t)b * rows_per_cta;
    const int64_t r1 = r0 + rows_per_cta < n ? r0 + rows_per_cta : n;
    const int c = t % TN_NC, jg = t / TN_NC;  // outputs (jg + 16 q, c), q = 0..3
    float2 acc[TN_JMAX / 16];
#pragma unroll
    for (int q = 0; q < TN_JMAX / 16; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int64_t rc = r0; rc < r1; rc += TN_TR) {
        for (int i = t; i < J * TN_TR; i += TN_THREADS) {
            const int j = i / TN_TR, k = i % TN_TR;
            const int64_t row = rc + k;
            Vs[j][k] = row < r1 ? ld_f2(V + j * sv + row) : make_float2(0.f, 0.f);
        }
        for (int i = t; i < TN_NC * TN_TR; i += TN_THREADS) {
            const int cc = i / TN_TR, k = i % TN_TR;
            const int64_t row = rc + k;
            Ws[cc][k] = (row < r1 && c0 + cc < N) ? ld_f2(W + (c0 + cc) * sw + row) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < TN_TR; ++k) {
            const float2 w = Ws[c][k];
#pragma unroll
            for (int q = 0; q < TN_JMAX / 16; ++q) {
                const int j = jg + 16 * q;
                if (j < J) {
                    const float2 v = Vs[j][k];  // conj(v) w
                    acc[q].x = fmaf(v.x, w.x, fmaf(v.y, w.y, acc[q].x));
                    acc[q].y = fmaf(v.x, w.y, fmaf(-v.y, w.x, acc[q].y));
                }
            }
        }
        __syncthreads();
    }
    if (c0 + c < N) {
#pragma unroll
        for (int q = 0; q < TN_JMAX / 16; ++q) {
            const int j = jg + 16 * q;
            if (j < J)
                partial[((int64_t)(c0 + c) * rstride + j) * nblk + b] =
                    make_double2((double)acc[q].x, (double)acc[q].y);
        }
    }
}

constexpr int NN_TR = 64;  // rows per CTA
constexpr int NN_NC = 32;  // columns per CTA (8 per thread)

// W_col[row] += alpha * sum_j V_j[row] C[col * cstride + j]  (C complex128, W complex128).
template <class TV>
__global__ void __launch_bounds__(TN_THREADS)
    k_tsmm_nn(const TV* __restrict__ V, int64_t sv, int J, const double2* __restrict__ C, int cstride,
              double2* __restrict__ W, int64_t sw, int N, int64_t n, double alpha) {
    __shared__ float2 Vs[TN_JMAX][NN_TR];
    __shared__ float2 Cs[TN_JMAX][NN_NC];
    const int t = threadIdx.x;
    const int64_t rbase = (int64_t)blockIdx.x * NN_TR;
    const int c0 = blockIdx.y * NN_NC;
    for (int i = t; i < J * NN_TR; i += TN_THREADS) {
        const int j = i / NN_TR, k = i % NN_TR;
        const int64_t row = rbase + k;
        Vs[j][k] = row < n ? ld_f2(V + j * sv + row) : make_float2(0.f, 0.f);
    }
    for (int i = t; i < J * NN_NC; i += TN_THREADS) {
        const int cc = i / J, j = i % J;
        Cs[j][cc] = c0 + cc < N ? ld_f2(C + (int64_t)(c0 + cc) * cstride + j) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int r = t % NN_TR, cg = t / NN_TR;  // row r, columns cg * 8 .. cg * 8 + 7 (one group per warp)
    float2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int j = 0; j < J; ++j) {
        const float2 v = Vs[j][r];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float2 cf = Cs[j][cg * 8 + q];
            acc[q].x = fmaf(v.x, cf.x, fmaf(-v.y, cf.y, acc[q].x));
            acc[q].y = fmaf(v.x, cf.y, fmaf(v.y, cf.x, acc[q].y));
        }
    }
    const int64_t row = rbase + r;
    if (row >= n) return;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int col = c0 + cg * 8 + q;
        if (col < N) {
            double2* p = W + col * sw + row;
            const double2 a = *p;
            *p = make_double2(a.x + alpha * (double)acc[q].x, a.y + alpha * (double)acc[q].y);
        }
    }
}

}  // namespace

template <class TV>
cudaError_t tsmm_tn(const TV* V, int64_t sv, int J, const double2* W, int64_t sw, int N, int64_t n,
                    const Reduce& rd, cudaStream_t st) {
    if (J < 1 || J > TN_JMAX || N < 1 || rd.stride < J) return cudaErrorInvalidValue;
    if ((int64_t)N > 65535 * (int64_t)TN_NC) return cudaErrorInvalidValue;
    const int64_t rows = (n + rd.nblk - 1) / rd.nblk;
    dim3 grid(rd.nblk, (N + TN_NC - 1) / TN_NC);
    k_tsmm_tn<TV><<<grid, TN_THREADS, 0, st>>>(V, sv, J, W, sw, N, n, rows, rd.partial, rd.stride, rd.nblk);
    count_launch();
    return cudaGetLastError();
}

template <class TV>
cudaError_t tsmm_nn(const TV* V, int64_t sv, int J, const double2* C, int cstride, double2* W, int64_t sw, int N,
                    int64_t n, double alpha, cudaStream_t st) {
    if (J < 1 || J > TN_JMAX || N < 1 || cstride < J) return cudaErrorInvalidValue;
    if ((int64_t)N > 65535 * (int64_t)NN_NC) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((n + NN_TR - 1) / NN_TR), (N + NN_NC - 1) / NN_NC);
    k_tsmm_nn<TV><<<grid, TN_THREADS, 0, st>>>(V, sv, J, C, cstride, W, sw, N, n, alpha);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t tsmm_tn<float2>(const float2*, int64_t, int, const double2*, int64_t, int, int64_t,
                                     const Reduce&, cudaStream_t);
template cudaError_t tsmm_nn<float2>(const float2*, int64_t, int, const double2*, int, double2*, int64_t, int,
                                     int64_t, double, cudaStream_t);

}  // namespace sgn
