// Tall-skinny vector kernels: multi-dot products with deterministic two-stage
// FP64 reductions, the fused passes of classical Gram-Schmidt with
// reorthogonalisation (CGS2) for the Arnoldi relation eq. (2.4), the basis
// update of Algorithm 1 and the LR projection r -> (I - R L^dag) r (Sec. 4).
//
// Element granularity is a 16-byte "pack": one complex128 or two complex64.
// A thread owns PKT packs of one column (PKT = 1, 2 or 4, a template
// parameter); a CTA of NT threads owns NT*PKT consecutive packs.  The number
// of CTAs per column is chosen so that the grid fills whole waves of the GPU
// (wave_blocks), and PKT follows from it.  Dot products: each thread forms its PKT pack products
// (in FP32 for complex64 storage, i.e. chunks of 8 complex products), promotes
// them to FP64 and the rest of the reduction -- warp shuffles, the CTA sum and
// the per-column sum over CTAs -- is FP64 in a fixed order (no atomics).
#include "blas.cuh"

#include <cstdlib>

#include <algorithm>

namespace sgn {
namespace {

constexpr int NT = 256;
constexpr int NWARP = NT / 32;
constexpr int PK = 4;  // default packs per thread (reduce_blocks)
constexpr int MAXSLOT = 136;  // >= 2 kmax + 3 (delayed CGS2), >= deflation size + 1, >= eigensolver block + 1

template <class T>
struct Ops;

template <>
struct Ops<double2> {
    using P = double2;
    using C = double2;  // coefficient type used in the arithmetic
    static constexpr int CPX = 1;
    static __device__ __forceinline__ P ld_ro(const double2* b, int64_t pk) { return __ldg(b + pk); }
    static __device__ __forceinline__ P ld(const double2* b, int64_t pk) { return b[pk]; }
    static __device__ __forceinline__ void st(double2* b, int64_t pk, P v) { b[pk] = v; }
    static __device__ __forceinline__ P zero() { return make_double2(0, 0); }
    static __device__ __forceinline__ C coef(double2 c) { return c; }
    // conj(v) * w
    static __device__ __forceinline__ double2 dot(P v, P w) { return cconjmul(v, w); }
    static __device__ __forceinline__ double nrm2(P w) { return w.x * w.x + w.y * w.y; }
    // w -= c v
    static __device__ __forceinline__ void sub_cv(P& w, C c, P v) {
        w.x = fma(-c.x, v.x, w.x);
        w.x = fma(c.y, v.y, w.x);
        w.y = fma(-c.x, v.y, w.y);
        w.y = fma(-c.y, v.x, w.y);
    }
    // a += c v
    static __device__ __forceinline__ void add_cv(P& a, C c, P v) {
        a.x = fma(c.x, v.x, a.x);
        a.x = fma(-c.y, v.y, a.x);
        a.y = fma(c.x, v.y, a.y);
        a.y = fma(c.y, v.x, a.y);
    }
    static __device__ __forceinline__ P scal(P v, double s) { return make_double2(v.x * s, v.y * s); }
    // x (complex128 array, CPX entries per pack) += v
    static __device__ __forceinline__ void add_to(double2* x, int64_t pk, P v) {
        double2 a = x[pk];
        x[pk] = make_double2(a.x + v.x, a.y + v.y);
    }
    // x += c v computed in FP64
    static __device__ __forceinline__ void add_cv_f64(double2 acc[1], double2 c, P v) {
        acc[0].x = fma(c.x, v.x, acc[0].x);
        acc[0].x = fma(-c.y, v.y, acc[0].x);
        acc[0].y = fma(c.x, v.y, acc[0].y);
        acc[0].y = fma(c.y, v.x, acc[0].y);
    }
};

template <>
struct Ops<float2> {
    using P = float4;
    using C = float2;
    static constexpr int CPX = 2;
    static __device__ __forceinline__ P ld_ro(const float2* b, int64_t pk) {
        return __ldg(reinterpret_cast<const float4*>(b) + pk);
    }
    static __device__ __forceinline__ P ld(const float2* b, int64_t pk) { return reinterpret_cast<const float4*>(b)[pk]; }
    static __device__ __forceinline__ void st(float2* b, int64_t pk, P v) { reinterpret_cast<float4*>(b)[pk] = v; }
    static __device__ __forceinline__ P zero() { return make_float4(0, 0, 0, 0); }
    static __device__ __forceinline__ C coef(double2 c) { return make_float2((float)c.x, (float)c.y); }
    static __device__ __forceinline__ double2 dot(P v, P w) {
        float re = v.x * w.x;
        re = fmaf(v.y, w.y, re);
        re = fmaf(v.z, w.z, re);
        re = fmaf(v.w, w.w, re);
        float im = v.x * w.y;
        im = fmaf(-v.y, w.x, im);
        im = fmaf(v.z, w.w, im);
        im = fmaf(-v.w, w.z, im);
        return make_double2(re, im);
    }
    static __device__ __forceinline__ double nrm2(P w) {
        float a = w.x * w.x;
        a = fmaf(w.y, w.y, a);
        a = fmaf(w.z, w.z, a);
        a = fmaf(w.w, w.w, a);
        return a;
    }
    // FP32 results: no FP64 instruction in the inner loops (FP64 runs at 1/64 rate)
    static __device__ __forceinline__ void dot_acc(float& re, float& im, P v, P w) {
        re = fmaf(v.x, w.x, re);
        re = fmaf(v.y, w.y, re);
        re = fmaf(v.z, w.z, re);
        re = fmaf(v.w, w.w, re);
        im = fmaf(v.x, w.y, im);
        im = fmaf(-v.y, w.x, im);
        im = fmaf(v.z, w.w, im);
        im = fmaf(-v.w, w.z, im);
    }
    static __device__ __forceinline__ void nrm2_acc(float& a, P w) {
        a = fmaf(w.x, w.x, a);
        a = fmaf(w.y, w.y, a);
        a = fmaf(w.z, w.z, a);
        a = fmaf(w.w, w.w, a);
    }
    static __device__ __forceinline__ P scalf(P v, float f) { return make_float4(v.x * f, v.y * f, v.z * f, v.w * f); }
    static __device__ __forceinline__ void sub_cv(P& w, C c, P v) {
        w.x = fmaf(-c.x, v.x, w.x);
        w.x = fmaf(c.y, v.y, w.x);
        w.y = fmaf(-c.x, v.y, w.y);
        w.y = fmaf(-c.y, v.x, w.y);
        w.z = fmaf(-c.x, v.z, w.z);
        w.z = fmaf(c.y, v.w, w.z);
        w.w = fmaf(-c.x, v.w, w.w);
        w.w = fmaf(-c.y, v.z, w.w);
    }
    static __device__ __forceinline__ void add_cv(P& a, C c, P v) {
        a.x = fmaf(c.x, v.x, a.x);
        a.x = fmaf(-c.y, v.y, a.x);
        a.y = fmaf(c.x, v.y, a.y);
        a.y = fmaf(c.y, v.x, a.y);
        a.z = fmaf(c.x, v.z, a.z);
        a.z = fmaf(-c.y, v.w, a.z);
        a.w = fmaf(c.x, v.w, a.w);
        a.w = fmaf(c.y, v.z, a.w);
    }
    static __device__ __forceinline__ P scal(P v, double s) {
        float f = (float)s;
        return make_float4(v.x * f, v.y * f, v.z * f, v.w * f);
    }
    static __device__ __forceinline__ void add_to(double2* x, int64_t pk, P v) {
        double2 a = x[2 * pk], b = x[2 * pk + 1];
        x[2 * pk] = make_double2(a.x + v.x, a.y + v.y);
        x[2 * pk + 1] = make_double2(b.x + v.z, b.y + v.w);
    }
    static __device__ __forceinline__ void add_cv_f64(double2 acc[2], double2 c, P v) {
        acc[0].x = fma(c.x, (double)v.x, acc[0].x);
        acc[0].x = fma(-c.y, (double)v.y, acc[0].x);
        acc[0].y = fma(c.x, (double)v.y, acc[0].y);
        acc[0].y = fma(c.y, (double)v.x, acc[0].y);
        acc[1].x = fma(c.x, (double)v.z, acc[1].x);
        acc[1].x = fma(-c.y, (double)v.w, acc[1].x);
        acc[1].y = fma(c.x, (double)v.w, acc[1].y);
        acc[1].y = fma(c.y, (double)v.z, acc[1].y);
    }
};

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Sum over the 32 lanes of an FP32 value kept as an unevaluated pair (hi, lo)
// (error-free TwoSum at every level): about FP64 accuracy for the tree at FP32
// instruction rates (FP64 runs at 1/64 of the FP32 rate on this part).
__device__ __forceinline__ float2 warp_sum_pair(float v) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        // TwoSum(hi, ohi) = (s, e) exactly, then FastTwoSum(s, e + lo + olo).  Written
        // with __fsub_rn: the same algebra spelled as __fadd_rn(x, -__fadd_rn(..))
        // was measured to lose the error term on this toolchain.
        const float s = __fadd_rn(hi, ohi);
        const float bp = __fsub_rn(s, hi);
        const float ap = __fsub_rn(s, bp);
        const float e = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(ohi, bp));
        const float t = __fadd_rn(e, __fadd_rn(lo, olo));
        const float nh = __fadd_rn(s, t);
        lo = __fsub_rn(t, __fsub_rn(nh, s));
        hi = nh;
    }
    return make_float2(hi, lo);
}
// Double-float sum of the 256 FP32 values st[0..255] (one per thread of the CTA)
// by one warp: 8 values per lane with TwoSum, then the lane butterfly.
__device__ __forceinline__ double cta_sum_df(const float* st, int lane) {
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int q = 0; q < NT / 32; ++q) {
        const float v = st[lane + 32 * q];
        const float s = __fadd_rn(hi, v);
        const float bp = __fsub_rn(s, hi);
        const float ap = __fsub_rn(s, bp);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(v, bp)));
        hi = s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = __fadd_rn(hi, ohi);
        const float bp = __fsub_rn(s, hi);
        const float ap = __fsub_rn(s, bp);
        const float e = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(ohi, bp));
        const float t = __fadd_rn(e, __fadd_rn(lo, olo));
        const float nh = __fadd_rn(s, t);
        lo = __fsub_rn(t, __fsub_rn(nh, s));
        hi = nh;
    }
    return (double)hi + (double)lo;
}

// Warp sums of a per-thread FP32 complex partial (re, im); lane 0 stores the
// FP64 result in sm[slot][warp].
__device__ __forceinline__ void warp_store_f(double2 (*sm)[NWARP], int slot, float re, float im, int lane, int warp) {
    const float2 r = warp_sum_pair(re);
    const float2 i = warp_sum_pair(im);
    if (lane == 0) sm[slot][warp] = make_double2((double)r.x + (double)r.y, (double)i.x + (double)i.y);
}

// Store the per-warp values sm[slot][warp] summed over warps into the partials.
__device__ __forceinline__ void flush_partials(double2 (*sm)[NWARP], int nslot, const Reduce& rd, int col) {
    __syncthreads();
    for (int j = threadIdx.x; j < nslot; j += NT) {
        double2 a = sm[j][0];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) a = cadd(a, sm[j][w]);
        rd.partial[((int64_t)col * rd.stride + j) * rd.nblk + blockIdx.x] = a;
    }
}

// ---------------------------------------------------------------- kernels --

// partial[j] = sum_e conj(V_j[e]) w[e], j < J; slot J: ||w||^2 if with_norm.
template <class T, int PKT>
__global__ void __launch_bounds__(NT) k_mdot(Basis<T> V, int J, const T* __restrict__ w, int64_t wsr, int64_t npk,
                                             Reduce rd, int with_norm, const int* __restrict__ skip) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    __shared__ double2 sm[MAXSLOT][NWARP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T* wc = w + col * wsr;
    const int64_t base = (int64_t)blockIdx.x * NT * PKT + threadIdx.x;
    typename O::P wv[PKT];
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        int64_t i = base + p * NT;
        wv[p] = i < npk ? O::ld_ro(wc, i) : O::zero();
    }
    const T* vb = V.base + col * V.sr;
    for (int j = 0; j < J; ++j) {
        const T* vj = vb + j * V.sj;
        if constexpr (O::CPX == 2) {
            float ax = 0.f, ay = 0.f;  // FP32 chunk of PKT packs (8 complex products)
#pragma unroll
            for (int p = 0; p < PKT; ++p) {
                int64_t i = base + p * NT;
                if (i < npk) O::dot_acc(ax, ay, O::ld_ro(vj, i), wv[p]);
            }
            warp_store_f(sm, j, ax, ay, lane, warp);
        } else {
            double2 acc = make_double2(0, 0);
#pragma unroll
            for (int p = 0; p < PKT; ++p) {
                int64_t i = base + p * NT;
                if (i < npk) acc = cadd(acc, O::dot(O::ld_ro(vj, i), wv[p]));
            }
            acc = warp_sum(acc);
            if (lane == 0) sm[j][warp] = acc;
        }
    }
    if (with_norm) {
        if constexpr (O::CPX == 2) {
            float a = 0.f;
#pragma unroll
            for (int p = 0; p < PKT; ++p) O::nrm2_acc(a, wv[p]);
            warp_store_f(sm, J, a, 0.f, lane, warp);
        } else {
            double a = 0;
#pragma unroll
            for (int p = 0; p < PKT; ++p) a += O::nrm2(wv[p]);
            double2 acc = warp_sum(make_double2(a, 0));
            if (lane == 0) sm[J][warp] = acc;
        }
    }
    flush_partials(sm, J + (with_norm ? 1 : 0), rd, col);
}

// w -= sum_j c_j V_j; then partial[j] = V_j^dag w (j < J) and slot J = ||w||^2.
template <class T, int PKT>
__global__ void __launch_bounds__(NT) k_maxpy_mdot(Basis<T> V, int J, const double2* __restrict__ coef, int cstride,
                                                   T* w, int64_t wsr, int64_t npk, Reduce rd,
                                                   const int* __restrict__ skip) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    __shared__ double2 sm[MAXSLOT][NWARP];
    __shared__ typename O::C cs[MAXSLOT];
    for (int j = threadIdx.x; j < J; j += NT) cs[j] = O::coef(coef[(int64_t)col * cstride + j]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* wc = w + col * wsr;
    const int64_t base = (int64_t)blockIdx.x * NT * PKT + threadIdx.x;
    typename O::P wv[PKT];
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        int64_t i = base + p * NT;
        wv[p] = i < npk ? O::ld(wc, i) : O::zero();
    }
    const T* vb = V.base + col * V.sr;
    for (int j = 0; j < J; ++j) {
        const T* vj = vb + j * V.sj;
        const typename O::C c = cs[j];
#pragma unroll
        for (int p = 0; p < PKT; ++p) {
            int64_t i = base + p * NT;
            if (i < npk) O::sub_cv(wv[p], c, O::ld_ro(vj, i));
        }
    }
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        int64_t i = base + p * NT;
        if (i < npk) O::st(wc, i, wv[p]);
    }
    for (int j = 0; j < J; ++j) {
        const T* vj = vb + j * V.sj;
        if constexpr (O::CPX == 2) {
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int p = 0; p < PKT; ++p) {
                int64_t i = base + p * NT;
                if (i < npk) O::dot_acc(ax, ay, O::ld_ro(vj, i), wv[p]);
            }
            warp_store_f(sm, j, ax, ay, lane, warp);
        } else {
            double2 acc = make_double2(0, 0);
#pragma unroll
            for (int p = 0; p < PKT; ++p) {
                int64_t i = base + p * NT;
                if (i < npk) acc = cadd(acc, O::dot(O::ld_ro(vj, i), wv[p]));
            }
            acc = warp_sum(acc);
            if (lane == 0) sm[j][warp] = acc;
        }
    }
    if constexpr (O::CPX == 2) {
        float a = 0.f;
#pragma unroll
        for (int p = 0; p < PKT; ++p) O::nrm2_acc(a, wv[p]);
        warp_store_f(sm, J, a, 0.f, lane, warp);
    } else {
        double a = 0;
#pragma unroll
        for (int p = 0; p < PKT; ++p) a += O::nrm2(wv[p]);
        double2 acc = warp_sum(make_double2(a, 0));
        if (lane == 0) sm[J][warp] = acc;
    }
    flush_partials(sm, J + 1, rd, col);
}

// out = (w - sum_j c_j V_j) * scale[col]   (out may alias w)
template <class T, int PKT>
__global__ void __launch_bounds__(NT) k_maxpy_scale(Basis<T> V, int J, const double2* __restrict__ coef, int cstride,
                                                    const T* w, int64_t wsr, T* out, int64_t osr,
                                                    const double* __restrict__ scale, int64_t npk,
                                                    const int* __restrict__ skip) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    __shared__ typename O::C cs[MAXSLOT];
    for (int j = threadIdx.x; j < J; j += NT) cs[j] = O::coef(coef[(int64_t)col * cstride + j]);
    __syncthreads();
    const T* wc = w + col * wsr;
    T* oc = out + col * osr;
    const double sc = scale ? scale[col] : 1.0;
    const int64_t base = (int64_t)blockIdx.x * NT * PKT + threadIdx.x;
    typename O::P wv[PKT];
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        int64_t i = base + p * NT;
        wv[p] = i < npk ? O::ld(wc, i) : O::zero();
    }
    const T* vb = V.base + col * V.sr;
    for (int j = 0; j < J; ++j) {
        const T* vj = vb + j * V.sj;
        const typename O::C c = cs[j];
#pragma unroll
        for (int p = 0; p < PKT; ++p) {
            int64_t i = base + p * NT;
            if (i < npk) O::sub_cv(wv[p], c, O::ld_ro(vj, i));
        }
    }
    if constexpr (O::CPX == 2) {
        const float scf = (float)sc;
#pragma unroll
        for (int p = 0; p < PKT; ++p) {
            int64_t i = base + p * NT;
            if (i < npk) O::st(oc, i, O::scalf(wv[p], scf));
        }
    } else {
#pragma unroll
        for (int p = 0; p < PKT; ++p) {
            int64_t i = base + p * NT;
            if (i < npk) O::st(oc, i, O::scal(wv[p], sc));
        }
    }
}

// x += sum_j c_j V_j in FP64 (x complex128), j < min(J, kk[col]).
template <class T, int PKT>
__global__ void __launch_bounds__(NT) k_update_x(Basis<T> V, int J, const double2* __restrict__ coef, int cstride,
                                                 double2* __restrict__ x, int64_t xsr, int64_t npk,
                                                 const int* __restrict__ skip, const int* __restrict__ kk) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    if (kk && kk[col] < J) J = kk[col];
    __shared__ double2 cs[MAXSLOT];
    for (int j = threadIdx.x; j < J; j += NT) cs[j] = coef[(int64_t)col * cstride + j];
    __syncthreads();
    double2* xc = x + col * xsr;
    const T* vb = V.base + col * V.sr;
    const int64_t base = (int64_t)blockIdx.x * NT * PKT + threadIdx.x;
    double2 acc[PKT][O::CPX];
#pragma unroll
    for (int p = 0; p < PKT; ++p)
#pragma unroll
        for (int q = 0; q < O::CPX; ++q) acc[p][q] = make_double2(0, 0);
    constexpr int UNR = 8 / PKT;
    for (int j0 = 0; j0 < J; j0 += UNR) {
        typename O::P q[UNR][PKT];
#pragma unroll
        for (int g = 0; g < UNR; ++g) {
            const T* vj = vb + (j0 + g) * V.sj;
#pragma unroll
            for (int p = 0; p < PKT; ++p) {
                const int64_t i = base + p * NT;
                q[g][p] = (j0 + g < J && i < npk) ? O::ld_ro(vj, i) : O::zero();
            }
        }
#pragma unroll
        for (int g = 0; g < UNR; ++g)
            if (j0 + g < J)
#pragma unroll
                for (int p = 0; p < PKT; ++p) O::add_cv_f64(acc[p], cs[j0 + g], q[g][p]);
    }
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        const int64_t i = base + p * NT;
        if (i >= npk) break;
#pragma unroll
        for (int q = 0; q < O::CPX; ++q) {
            double2 a = xc[i * O::CPX + q];
            xc[i * O::CPX + q] = make_double2(a.x + acc[p][q].x, a.y + acc[p][q].y);
        }
    }
}

// xs[i] += sum_j y_ij V_j for every shift i.  Each CTA takes one group of SG shifts for one
// tile of elements; the groups of a tile are consecutive CTAs (blockIdx.x = tile * ngrp + group),
// so they run together and the tile of V comes from HBM once, the other groups reading it from L2.
// SG = 2 by default (on the 10^4 workload 176 us per launch, against 193 us with SG = 4 and 253 us
// with SG = 8); with SG = 20 (all of the workloads' 20 poles in one CTA) the FP32 kernel needs 192
// registers and ran at half the speed.  Products and the sum over j in the
// storage precision; the add to xs in FP64.
template <class T, int SG>
__global__ void __launch_bounds__(NT) k_update_shifts(Basis<T> V, int J, const double2* __restrict__ y, int s,
                                                      int kmax, double2* __restrict__ xs, int64_t xs_shift,
                                                      int64_t xs_col, int64_t npk, const int* __restrict__ skip,
                                                      const int* __restrict__ kk) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    if (kk && kk[col] < J) J = kk[col];
    const int ngrp = (s + SG - 1) / SG;
    const int64_t tile = blockIdx.x / (unsigned)ngrp;
    const int g0 = (int)(blockIdx.x - tile * ngrp) * SG;
    const int ng = (s - g0) < SG ? (s - g0) : SG;
    extern __shared__ unsigned char smraw[];
    typename O::C* ys = reinterpret_cast<typename O::C*>(smraw);  // [ng][J]: this CTA's shifts
    for (int t = threadIdx.x; t < ng * J; t += NT) {
        int i = t / J, j = t % J;
        ys[t] = O::coef(y[((int64_t)col * s + g0 + i) * kmax + j]);
    }
    __syncthreads();
    const int64_t i = tile * NT + threadIdx.x;
    if (i >= npk) return;
    const T* vb = V.base + col * V.sr;
    {
        typename O::P acc[SG];
#pragma unroll
        for (int g = 0; g < SG; ++g) acc[g] = O::zero();
        // loads of 4 basis vectors in flight together
        for (int j0 = 0; j0 < J; j0 += 4) {
            typename O::P v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = j0 + u < J ? O::ld_ro(vb + (j0 + u) * V.sj, i) : O::zero();
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < J)
#pragma unroll
                    for (int g = 0; g < SG; ++g)
                        if (g < ng) O::add_cv(acc[g], ys[g * J + j0 + u], v[u]);
        }
#pragma unroll
        for (int g = 0; g < SG; ++g)
            if (g < ng) O::add_to(xs + (int64_t)(g0 + g) * xs_shift + col * xs_col, i, acc[g]);
    }
}

// Delayed CGS2, fused reduction of step j (Q = V_0..V_{J-1} orthonormal, u the
// once-orthogonalised candidate, z = A^2 u):  slots [0,J) s = Q^dag u,
// [J,2J) t = Q^dag z, 2J: u^dag u, 2J+1: u^dag z, 2J+2: z^dag z.  With z = null
// (the closing pass of a cycle) only s and u^dag u (slot J).
template <class T, int PKT>
__global__ void __launch_bounds__(NT) k_dcgs_dots(Basis<T> V, int J, const T* __restrict__ u,
                                                  const T* __restrict__ z, int64_t wsr, int64_t npk, Reduce rd,
                                                  const int* __restrict__ skip) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T* uc = u + col * wsr;
    const T* zc = z ? z + col * wsr : nullptr;
    const int64_t base = (int64_t)blockIdx.x * NT * PKT + threadIdx.x;
    typename O::P uv[PKT], zv[PKT];
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        int64_t i = base + p * NT;
        uv[p] = i < npk ? O::ld(uc, i) : O::zero();
        zv[p] = (zc && i < npk) ? O::ld(zc, i) : O::zero();
    }
    const T* vb = V.base + col * V.sr;
    if constexpr (O::CPX == 2) {
        // FP32 storage: per-thread FP32 chunk partials are staged in shared memory
        // for a tile of TL basis vectors; each (vector, component) slot is then summed
        // over the whole CTA by one warp in double-float and written as this CTA's
        // FP64 partial.  Four values per vector: Re/Im of q^dag u and of q^dag z.
        constexpr int TL = 8;
        __shared__ float st[TL * 4][NT + 8];  // rows padded: the segmented sums below are bank-conflict free
        double* pd = reinterpret_cast<double*>(rd.partial);
        auto put = [&](int slot, int comp, double v) {
            pd[2 * (((int64_t)col * rd.stride + slot) * rd.nblk + blockIdx.x) + comp] = v;
        };
        const int nv = zc ? 4 : 2;
        // loads of GB basis vectors are issued together: 8 independent 16-byte
        // loads in flight per thread (4 with PKT = 4, whose registers hold 4 packs
        // of u and z already)
        constexpr int GB = PKT == 4 ? 1 : 8 / PKT;
        for (int l0 = 0; l0 < J; l0 += TL) {
            const int tl = (J - l0) < TL ? (J - l0) : TL;
#pragma unroll
            for (int g0 = 0; g0 < TL; g0 += GB) {
                if (g0 >= tl) break;
                typename O::P q[GB][PKT];
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    const T* vl = vb + (l0 + g0 + g) * V.sj;
#pragma unroll
                    for (int p = 0; p < PKT; ++p) {
                        const int64_t i = base + p * NT;
                        q[g][p] = (g0 + g < tl && i < npk) ? O::ld_ro(vl, i) : O::zero();
                    }
                }
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    if (g0 + g < tl) {
                        float sx = 0.f, sy = 0.f, tx = 0.f, ty = 0.f;
#pragma unroll
                        for (int p = 0; p < PKT; ++p) {
                            O::dot_acc(sx, sy, q[g][p], uv[p]);
                            if (zc) O::dot_acc(tx, ty, q[g][p], zv[p]);
                        }
                        st[(g0 + g) * 4 + 0][threadIdx.x] = sx;
                        st[(g0 + g) * 4 + 1][threadIdx.x] = sy;
                        st[(g0 + g) * 4 + 2][threadIdx.x] = tx;
                        st[(g0 + g) * 4 + 3][threadIdx.x] = ty;
                    }
                }
            }
            __syncthreads();
            {
                // slot sl = tid / 8 (TL * 4 = 32 slots for 256 threads), summed by 8 lanes:
                // lane seg adds values seg, seg + 8, ... in FP32, then a 3-level shuffle
                // tree.  Every partial is a sum of at most a few hundred FP32 products
                // (error ~ eps_32 times the sum of their moduli, the rounding the FP32
                // products carry anyway); the sum over CTAs is FP64.
                static_assert(TL * 4 * 8 == NT, "one 8-lane group per slot");
                const int sl = threadIdx.x >> 3, seg = threadIdx.x & 7;
                float a = 0.f;
#pragma unroll
                for (int k = 0; k < NT / 8; ++k) a += st[sl][k * 8 + seg];
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                a += __shfl_xor_sync(0xffffffffu, a, 4);
                const int g = sl >> 2, v = sl & 3;
                if (seg == 0 && g < tl && v < nv) put(v < 2 ? l0 + g : J + l0 + g, v & 1, (double)a);
            }
            __syncthreads();
        }
        // norms and u^dag z
        float a = 0.f, bx = 0.f, by = 0.f, gz = 0.f;
#pragma unroll
        for (int p = 0; p < PKT; ++p) {
            O::nrm2_acc(a, uv[p]);
            if (zc) {
                O::dot_acc(bx, by, uv[p], zv[p]);
                O::nrm2_acc(gz, zv[p]);
            }
        }
        st[0][threadIdx.x] = a;
        st[1][threadIdx.x] = bx;
        st[2][threadIdx.x] = by;
        st[3][threadIdx.x] = gz;
        __syncthreads();
        const int bs = zc ? 2 * J : J;
        if (warp < (zc ? 4 : 1)) {
            const double r = cta_sum_df(st[warp], lane);
            if (lane == 0) {
                if (warp == 0) {
                    put(bs, 0, r);
                    put(bs, 1, 0.0);
                } else if (warp == 1) {
                    put(bs + 1, 0, r);
                } else if (warp == 2) {
                    put(bs + 1, 1, r);
                } else {
                    put(bs + 2, 0, r);
                    put(bs + 2, 1, 0.0);
                }
            }
        }
        return;
    } else {
        // FP64 storage: the same tiling with FP64 values; each (vector, component)
        // slot is summed over the CTA by one warp in a fixed order (8 values per
        // lane, then a shuffle tree), one warp-reduction per slot instead of one per
        // warp and vector.
        constexpr int TL = 4;
        __shared__ double sd[TL * 4][NT];
        double* pd = reinterpret_cast<double*>(rd.partial);
        auto put = [&](int slot, int comp, double v) {
            pd[2 * (((int64_t)col * rd.stride + slot) * rd.nblk + blockIdx.x) + comp] = v;
        };
        auto cta_sum = [&](const double* row) {
            double a = 0;
#pragma unroll
            for (int k = 0; k < NT / 32; ++k) a += row[lane + 32 * k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            return a;
        };
        const int nv = zc ? 4 : 2;
        constexpr int GB = PKT == 4 ? 1 : 4 / PKT;
        for (int l0 = 0; l0 < J; l0 += TL) {
            const int tl = (J - l0) < TL ? (J - l0) : TL;
#pragma unroll
            for (int g0 = 0; g0 < TL; g0 += GB) {
                if (g0 >= tl) break;
                typename O::P q[GB][PKT];
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    const T* vl = vb + (l0 + g0 + g) * V.sj;
#pragma unroll
                    for (int p = 0; p < PKT; ++p) {
                        const int64_t i = base + p * NT;
                        q[g][p] = (g0 + g < tl && i < npk) ? O::ld_ro(vl, i) : O::zero();
                    }
                }
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    if (g0 + g < tl) {
                        double2 as = make_double2(0, 0), at = make_double2(0, 0);
#pragma unroll
                        for (int p = 0; p < PKT; ++p) {
                            as = cadd(as, O::dot(q[g][p], uv[p]));
                            if (zc) at = cadd(at, O::dot(q[g][p], zv[p]));
                        }
                        sd[(g0 + g) * 4 + 0][threadIdx.x] = as.x;
                        sd[(g0 + g) * 4 + 1][threadIdx.x] = as.y;
                        sd[(g0 + g) * 4 + 2][threadIdx.x] = at.x;
                        sd[(g0 + g) * 4 + 3][threadIdx.x] = at.y;
                    }
                }
            }
            __syncthreads();
            for (int sl = warp; sl < tl * 4; sl += NWARP) {
                const int g = sl >> 2, v = sl & 3;
                if (v >= nv) continue;
                const double r = cta_sum(sd[sl]);
                if (lane == 0) put(v < 2 ? l0 + g : J + l0 + g, v & 1, r);
            }
            __syncthreads();
        }
        // norms and u^dag z
        double a = 0, bx = 0, by = 0, gz = 0;
#pragma unroll
        for (int p = 0; p < PKT; ++p) {
            a += O::nrm2(uv[p]);
            if (zc) {
                const double2 d = O::dot(uv[p], zv[p]);
                bx += d.x;
                by += d.y;
                gz += O::nrm2(zv[p]);
            }
        }
        sd[0][threadIdx.x] = a;
        sd[1][threadIdx.x] = bx;
        sd[2][threadIdx.x] = by;
        sd[3][threadIdx.x] = gz;
        __syncthreads();
        const int bs = zc ? 2 * J : J;
        if (warp < (zc ? 4 : 1)) {
            const double r = cta_sum(sd[warp]);
            if (lane == 0) {
                if (warp == 0) {
                    put(bs, 0, r);
                    put(bs, 1, 0.0);
                } else if (warp == 1) {
                    put(bs + 1, 0, r);
                } else if (warp == 2) {
                    put(bs + 1, 1, r);
                } else {
                    put(bs + 2, 0, r);
                    put(bs + 2, 1, 0.0);
                }
            }
        }
    }
}

// Delayed CGS2, update of step j:  q_j = (u - Q s) / rho  (written over u), and
// the next candidate  u_{j+1} = z / rho - Q c - d q_j  (when next != null).
// Coefficients per column: [0,J) s, [J,2J) c, 2J: (1/rho, 0), 2J+1: d.
template <class T, int PKT>
__global__ void __launch_bounds__(NT) k_dcgs_update(Basis<T> V, int J, const double2* __restrict__ coef,
                                                    int cstride, T* u, const T* __restrict__ z, T* next,
                                                    int64_t wsr, int64_t npk, const int* __restrict__ skip) {
    using O = Ops<T>;
    const int col = blockIdx.y;
    if (skip && skip[col]) return;
    __shared__ typename O::C cs[MAXSLOT], cc[MAXSLOT];
    __shared__ double ex[2][2];
    const double2* cf = coef + (int64_t)col * cstride;
    for (int l = threadIdx.x; l < J; l += NT) {
        cs[l] = O::coef(cf[l]);
        cc[l] = O::coef(cf[J + l]);
    }
    if (threadIdx.x == 0) {
        ex[0][0] = cf[2 * J].x;
        ex[1][0] = cf[2 * J + 1].x;
        ex[1][1] = cf[2 * J + 1].y;
    }
    __syncthreads();
    const double inv_rho = ex[0][0];
    const float inv_rho_f = (float)inv_rho;
    const typename O::C dd = O::coef(make_double2(ex[1][0], ex[1][1]));
    T* uc = u + col * wsr;
    const T* zc = next ? z + col * wsr : nullptr;
    T* nc = next ? next + col * wsr : nullptr;
    const T* vb = V.base + col * V.sr;
    const int64_t base = (int64_t)blockIdx.x * NT * PKT + threadIdx.x;
    // Q s and Q c with the basis loop outside: the loads of UNR basis vectors
    // (PKT packs each) are independent and in flight together
    typename O::P qs[PKT], qc[PKT];
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        qs[p] = O::zero();
        qc[p] = O::zero();
    }
    constexpr int UNR = 8 / PKT;
    for (int l0 = 0; l0 < J; l0 += UNR) {
        typename O::P q[UNR][PKT];
#pragma unroll
        for (int g = 0; g < UNR; ++g) {
            const T* vl = vb + (l0 + g) * V.sj;
#pragma unroll
            for (int p = 0; p < PKT; ++p) {
                const int64_t i = base + p * NT;
                q[g][p] = (l0 + g < J && i < npk) ? O::ld_ro(vl, i) : O::zero();
            }
        }
#pragma unroll
        for (int g = 0; g < UNR; ++g) {
            if (l0 + g < J) {
                const typename O::C a = cs[l0 + g], c = cc[l0 + g];
#pragma unroll
                for (int p = 0; p < PKT; ++p) {
                    O::add_cv(qs[p], a, q[g][p]);
                    if (nc) O::add_cv(qc[p], c, q[g][p]);
                }
            }
        }
    }
    typename O::C one;
    if constexpr (O::CPX == 1) {
        one = make_double2(1.0, 0.0);
    } else {
        one = make_float2(1.0f, 0.0f);
    }
#pragma unroll
    for (int p = 0; p < PKT; ++p) {
        const int64_t i = base + p * NT;
        if (i >= npk) break;
        typename O::P uv = O::ld(uc, i);
        // q_j = (u - qs) / rho
        O::sub_cv(uv, one, qs[p]);
        typename O::P qj;
        if constexpr (O::CPX == 2) {
            qj = O::scalf(uv, inv_rho_f);
        } else {
            qj = O::scal(uv, inv_rho);
        }
        O::st(uc, i, qj);
        if (nc) {
            typename O::P nv;
            if constexpr (O::CPX == 2) {
                nv = O::scalf(O::ld(zc, i), inv_rho_f);
            } else {
                nv = O::scal(O::ld(zc, i), inv_rho);
            }
            O::sub_cv(nv, one, qc[p]);
            O::sub_cv(nv, dd, qj);
            O::st(nc, i, nv);
        }
    }
}

// Second stage of every reduction plus the scalar bookkeeping that consumes it.
// The scalar work of a reduction once the slot sums of column col are known
// (sums: shared memory, nslot entries).  Called by every thread of one CTA.
__device__ void reduce_tail(const double2* sums, int col, int nslot, int mode, int colidx, const DevState& S,
                            const double2* __restrict__ lambda) {
    __shared__ double2 gsh[MAXSLOT];
    const int64_t cr = (int64_t)col * S.rstride;
    switch (mode) {
        case RM_STORE:
            for (int j = threadIdx.x; j < nslot; j += NT) S.red[cr + j] = sums[j];
            break;
        case RM_SIGNED:
            for (int j = threadIdx.x; j < nslot; j += NT) {
                double sg = lambda[j].x > 0 ? 1.0 : -1.0;
                S.red[cr + j] = make_double2(sg * sums[j].x, sg * sums[j].y);
            }
            break;
        case RM_H1:
            for (int j = threadIdx.x; j < nslot - 1; j += NT) S.h1[cr + j] = sums[j];
            if (threadIdx.x == 0) S.norm0[col] = sqrt(sums[nslot - 1].x);
            break;
        case RM_P2: {
            const int J = nslot - 1;  // = colidx + 1
            const int64_t hb = (int64_t)col * (S.kmax + 1) * S.kmax;
            for (int l = threadIdx.x; l < J; l += NT) {
                S.red[cr + l] = sums[l];
                S.H[hb + (int64_t)l * S.kmax + colidx] = cadd(S.h1[cr + l], sums[l]);
            }
            if (threadIdx.x == 0) {
                double h2 = 0;
                for (int l = 0; l < J; ++l) h2 += cabs2(sums[l]);
                double hn2 = sums[J].x - h2;
                double hn = hn2 > 0 ? sqrt(hn2) : 0.0;
                S.H[hb + (int64_t)(colidx + 1) * S.kmax + colidx] = make_double2(hn, 0);
                if (!(hn > S.bd_tol * S.norm0[col])) {
                    S.kk[col] = colidx + 1;
                    S.skip[col] = 1;
                    S.scale[col] = 0;
                    if (!isfinite(hn2)) atomicOr(S.err, 2);
                } else {
                    S.scale[col] = 1.0 / hn;
                }
            }
            break;
        }
        case RM_DCGS:
        case RM_DCGS_FINAL: {
            // Delayed CGS2 bookkeeping of step j = colidx (see k_dcgs_dots for the slots).
            const int j = colidx;
            const bool fin = mode == RM_DCGS_FINAL;
            const int64_t hb = (int64_t)col * (S.kmax + 1) * S.kmax;
            const int km = S.kmax;
            double2* H = S.H + hb;
            const double2 alpha = sums[fin ? j : 2 * j];
            __shared__ double rho_sh;
            __shared__ int broke_sh;
            __shared__ double2 st_sh;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (warp == 0) {
                // s2 = sum_l |s_l|^2 and st = sum_l conj(s_l) t_l, l < j: lanes over l, fixed-order tree
                double2 s2v = make_double2(0, 0), st = make_double2(0, 0);
                for (int l = lane; l < j; l += 32) {
                    s2v.x += cabs2(sums[l]);
                    if (!fin) st = cadd(st, cconjmul(sums[l], sums[j + l]));
                }
                s2v = warp_sum(s2v);
                st = warp_sum(st);
                if (lane == 0) {
                    st_sh = st;
                    const double s2 = s2v.x;
                    double r2 = alpha.x - s2;
                    double rho = r2 > 0 ? sqrt(r2) : 0.0;
                    int broke = 0;
                    if (j == 0) {
                        S.beta[col] = rho;
                        broke = !(rho > 0);
                    } else {
                        broke = !(rho > S.bd_tol * S.norm0[col]);
                        H[(int64_t)j * km + (j - 1)] = make_double2(rho, 0);
                    }
                    if (!isfinite(r2)) {
                        atomicOr(S.err, 2);
                        broke = 1;
                    }
                    rho_sh = rho;
                    broke_sh = broke;
                }
            }
            __syncthreads();
            // correct column j-1: H[0:j, j-1] += s
            for (int l = threadIdx.x; l < j; l += NT) {
                double2 h = H[(int64_t)l * km + (j - 1)];
                H[(int64_t)l * km + (j - 1)] = cadd(h, sums[l]);
            }
            __syncthreads();
            const double rho = rho_sh;
            const int64_t cr = (int64_t)col * S.rstride;
            if (fin) {
                // closing pass: q_k = (u - Q s) / rho; an invariant Krylov space (rho ~ 0)
                // leaves q_k = 0, so the restart norm is 0 and the column converges
                for (int l = threadIdx.x; l < j; l += NT) S.red[cr + l] = sums[l];
                if (threadIdx.x == 0) S.red[cr + 2 * j] = make_double2(broke_sh ? 0.0 : 1.0 / rho, 0);
                break;
            }
            if (broke_sh) {  // the Krylov space is invariant: FOM on its j columns is exact
                if (threadIdx.x == 0) {
                    S.kk[col] = j;
                    S.skip[col] = 1;
                }
                break;
            }
            for (int l = threadIdx.x; l < j; l += NT) S.red[cr + l] = sums[l];  // s
            // g = Hbar s, Hbar = H[0:j+1, 0:j]: warp w takes rows w, w + 8, ...; lanes split the
            // row (l = lane, lane + 32); every H load of the warp is issued before the sums
            if (j <= 64) {
                constexpr int RPW = (65 + NWARP - 1) / NWARP;
                double2 hv[RPW][2];
#pragma unroll
                for (int r = 0; r < RPW; ++r)
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int i = warp + r * NWARP, l = lane + 32 * q;
                        hv[r][q] = (i <= j && l < j && l >= i - 1) ? H[(int64_t)i * km + l] : make_double2(0, 0);
                    }
                const double2 s0 = lane < j ? sums[lane] : make_double2(0, 0);
                const double2 s1 = lane + 32 < j ? sums[lane + 32] : make_double2(0, 0);
#pragma unroll
                for (int r = 0; r < RPW; ++r) {
                    const int i = warp + r * NWARP;
                    if (i > j) break;  // uniform over the warp
                    const double2 g = warp_sum(cadd(cmul(hv[r][0], s0), cmul(hv[r][1], s1)));
                    if (lane == 0) gsh[i] = g;
                }
            } else {
                for (int i = threadIdx.x; i <= j; i += NT) {
                    double2 g = make_double2(0, 0);
                    for (int l = (i > 0 ? i - 1 : 0); l < j; ++l) g = cadd(g, cmul(H[(int64_t)i * km + l], sums[l]));
                    gsh[i] = g;
                }
            }
            __syncthreads();
            const double ir = 1.0 / rho;
            for (int i = threadIdx.x; i < j; i += NT) {
                double2 t = sums[j + i];
                double2 hp = make_double2((t.x - gsh[i].x) * ir, (t.y - gsh[i].y) * ir);
                H[(int64_t)i * km + j] = hp;                                             // tentative column j
                S.red[cr + j + i] = make_double2(gsh[i].x * ir + hp.x, gsh[i].y * ir + hp.y);  // c
            }
            if (threadIdx.x == 0) {
                const double2 st = st_sh;
                double2 beta = sums[2 * j + 1];
                double2 hjj = make_double2(((beta.x - st.x) * ir - gsh[j].x) * ir, ((beta.y - st.y) * ir - gsh[j].y) * ir);
                H[(int64_t)j * km + j] = hjj;
                S.red[cr + 2 * j] = make_double2(ir, 0);
                S.red[cr + 2 * j + 1] = make_double2(gsh[j].x * ir + hjj.x, gsh[j].y * ir + hjj.y);  // d
                S.norm0[col] = sqrt(sums[2 * j + 2].x) * ir;  // ~ ||A^2 q_j|| for the next breakdown test
            }
            break;
        }
        case RM_BETA_FIRST:
            if (threadIdx.x == 0) {
                double beta = sqrt(sums[0].x);
                S.beta[col] = beta;
                S.bnorm[col] = beta;
                S.kk[col] = S.kmax;
                for (int i = 0; i < S.s; ++i) S.rho[(int64_t)col * S.s + i] = make_double2(1, 0);
                if (!isfinite(beta)) atomicOr(S.err, 2);
                if (beta > 0 && isfinite(beta)) {
                    S.scale[col] = 1.0 / beta;
                    S.resest[col] = 1.0;
                    S.skip[col] = 0;
                    S.done[col] = 0;
                } else {
                    S.scale[col] = 0;
                    S.resest[col] = 0;
                    S.skip[col] = 1;
                    S.done[col] = 1;
                }
            }
            break;
        case RM_BETA_RESTART:
            if (threadIdx.x == 0) {
                if (S.kk[col] < S.kmax) {  // invariant subspace met: FOM is exact
                    S.resest[col] = 0;
                    S.done[col] = 1;
                    S.skip[col] = 1;
                    S.scale[col] = 0;
                    break;
                }
                double beta = sqrt(sums[0].x);
                double rmax = 0;
                for (int i = 0; i < S.s; ++i) {
                    double2 r = S.rho[(int64_t)col * S.s + i];
                    double a = sqrt(cabs2(r)) * beta / S.bnorm[col];
                    rmax = a > rmax ? a : rmax;
                }
                S.beta[col] = beta;
                S.resest[col] = rmax;
                if (!isfinite(rmax)) {
                    atomicOr(S.err, 2);
                    S.done[col] = 1;
                    S.skip[col] = 1;
                    S.scale[col] = 0;
                    break;
                }
                const int conv = rmax <= S.tol || beta == 0;
                S.done[col] = conv;
                S.skip[col] = conv;
                S.scale[col] = beta > 0 ? 1.0 / beta : 0.0;
            }
            break;
    }
}

__global__ void __launch_bounds__(NT) k_reduce(Reduce rd, int nslot, int mode, int colidx, DevState S,
                                               const double2* __restrict__ lambda) {
    const int col = blockIdx.x;
    // RM_BETA_FIRST starts a solve; RM_BETA_RESTART must still see columns that
    // broke down in this cycle; every other mode is column work proper.
    if (mode == RM_BETA_RESTART && S.done[col]) return;
    if (mode != RM_BETA_FIRST && mode != RM_BETA_RESTART && S.skip[col]) return;
    __shared__ double2 sums[MAXSLOT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < nslot; j += NWARP) {
        const double2* p = rd.partial + ((int64_t)col * rd.stride + j) * rd.nblk;
        double2 a = make_double2(0, 0);
        // unrolled so that the loads of up to 8 partials per lane are in flight together
        // (the sum order, b = lane, lane + 32, ..., is fixed either way)
#pragma unroll 8
        for (int b = lane; b < rd.nblk; b += 32) a = cadd(a, p[b]);
        a = warp_sum(a);
        if (lane == 0) sums[j] = a;
    }
    __syncthreads();
    reduce_tail(sums, col, nslot, mode, colidx, S, lambda);
}

// Split form: CTA (col, g) sums slots g * NWARP .. g * NWARP + NWARP - 1 (one warp each,
// the same fixed order as k_reduce) into S.sums; the last CTA of the column to
// arrive loads all sums and does the scalar work.  Results are identical to
// k_reduce's whatever the arrival order.
__global__ void __launch_bounds__(NT) k_reduce_split(Reduce rd, int nslot, int mode, int colidx, DevState S,
                                                     const double2* __restrict__ lambda) {
    const int col = blockIdx.x;
    if (mode == RM_BETA_RESTART && S.done[col]) return;
    if (mode != RM_BETA_FIRST && mode != RM_BETA_RESTART && S.skip[col]) return;
    __shared__ double2 sums[MAXSLOT];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cr = (int64_t)col * S.rstride;
    const int j = blockIdx.y * NWARP + warp;
    if (j < nslot) {
        const double2* p = rd.partial + ((int64_t)col * rd.stride + j) * rd.nblk;
        double2 a = make_double2(0, 0);
#pragma unroll 8
        for (int b = lane; b < rd.nblk; b += 32) a = cadd(a, p[b]);
        a = warp_sum(a);
        if (lane == 0) S.sums[cr + j] = a;
    }
    __threadfence();  // this CTA's sums are visible device-wide before it is counted
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&S.rcount[col], 1) == (int)gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < nslot; i += NT) sums[i] = __ldcg(S.sums + cr + i);  // from L2, not a stale L1
    if (threadIdx.x == 0) S.rcount[col] = 0;  // ready for the next launch
    __syncthreads();
    reduce_tail(sums, col, nslot, mode, colidx, S, lambda);
}

// out = a x + b y + c z on whole blocks (real coefficients; z may be null).
template <class T>
__global__ void __launch_bounds__(NT) k_axpby3(T* __restrict__ out, double a, const T* __restrict__ x, double b,
                                               const T* __restrict__ y, double c, const T* __restrict__ z,
                                               int64_t npk) {
    using O = Ops<T>;
    const float af = (float)a, bf = (float)b, cf = (float)c;  // FP32 path: convert once
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < npk; i += (int64_t)gridDim.x * NT) {
        typename O::P r;
        if constexpr (O::CPX == 1) {
            typename O::P v = O::scal(O::ld(x, i), a);
            typename O::P w = O::scal(O::ld(y, i), b);
            r = make_double2(v.x + w.x, v.y + w.y);
            if (z) {
                typename O::P u = O::scal(O::ld(z, i), c);
                r = make_double2(r.x + u.x, r.y + u.y);
            }
        } else {
            typename O::P v = O::scalf(O::ld(x, i), af);
            typename O::P w = O::scalf(O::ld(y, i), bf);
            r = make_float4(v.x + w.x, v.y + w.y, v.z + w.z, v.w + w.w);
            if (z) {
                typename O::P u = O::scalf(O::ld(z, i), cf);
                r = make_float4(r.x + u.x, r.y + u.y, r.z + u.z, r.w + u.w);
            }
        }
        O::st(out, i, r);
    }
}

// Z_j = sum_i C[i][j] Y_i  (Y: q fields, Z: r fields, each n complex apart; C row-major q x r),
// SG output fields per sweep of Y.
constexpr int SG = 8;
template <class T>
__global__ void __launch_bounds__(NT) k_block_combine(const T* __restrict__ Y, int q, const double2* __restrict__ Cm,
                                                      int r, T* __restrict__ Z, int64_t n, int64_t npk) {
    using O = Ops<T>;
    __shared__ typename O::C cs[MAXSLOT * SG];
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    for (int g0 = 0; g0 < r; g0 += SG) {
        const int ng = (r - g0) < SG ? (r - g0) : SG;
        __syncthreads();
        for (int t = threadIdx.x; t < q * SG; t += NT) {
            int a = t / SG, g = t % SG;
            cs[t] = g < ng ? O::coef(Cm[(int64_t)a * r + g0 + g]) : O::coef(make_double2(0, 0));
        }
        __syncthreads();
        if (i < npk) {
            typename O::P acc[SG];
#pragma unroll
            for (int g = 0; g < SG; ++g) acc[g] = O::zero();
            for (int a = 0; a < q; ++a) {
                typename O::P v = O::ld_ro(Y + a * n, i);
#pragma unroll
                for (int g = 0; g < SG; ++g) O::add_cv(acc[g], cs[a * SG + g], v);
            }
#pragma unroll
            for (int g = 0; g < SG; ++g)
                if (g < ng) O::st(Z + (int64_t)(g0 + g) * n, i, acc[g]);
        }
    }
}

// Counter-based Gaussian start vectors: SplitMix64 of (seed, index), Box-Muller.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}
template <class T>
__global__ void k_random_fill(T* out, int64_t count, uint64_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t h1 = splitmix64(seed ^ (2 * (uint64_t)i)), h2 = splitmix64(seed ^ (2 * (uint64_t)i + 1));
        double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);
        double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
        double rr = sqrt(-2.0 * log(u1));
        double re = rr * cos(6.283185307179586 * u2), im = rr * sin(6.283185307179586 * u2);
        if constexpr (sizeof(T) == 16) {
            out[i] = T{re, im};
        } else {
            out[i] = T{(float)re, (float)im};
        }
    }
}

__global__ void k_f64_to_f32(const double2* __restrict__ in, float2* __restrict__ out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = in[i];
        out[i] = make_float2((float)v.x, (float)v.y);
    }
}
__global__ void k_f32_to_f64(const float2* __restrict__ in, double2* __restrict__ out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = in[i];
        out[i] = make_double2(v.x, v.y);
    }
}
__global__ void k_f64_to_bf16(const double2* __restrict__ in, __nv_bfloat162* __restrict__ out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = in[i];
        out[i] = __floats2bfloat162_rn((float)v.x, (float)v.y);
    }
}
// FP16 links: SU(3) entries have modulus <= 1, inside FP16's normal range (one rounding
// from FP32; entries below 6e-5 in modulus lose relative precision as subnormals, which
// costs at most 6e-8 absolute per entry)
__global__ void k_f64_to_f16(const double2* __restrict__ in, __half2* __restrict__ out, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = in[i];
        out[i] = __floats2half2_rn((float)v.x, (float)v.y);
    }
}

// r_j += sigma_j d_j - w_j for nb systems: r_j at r + roff[j] (complex128), w_j = A^2 d_j
// in FP32 and d_j in FP64, both at j * n.
__global__ void k_correct_residuals(double2* __restrict__ r, const long long* __restrict__ roff,
                                    const double* __restrict__ sig, const float2* __restrict__ w,
                                    const double2* __restrict__ d, int64_t n) {
    const int j = blockIdx.y;
    double2* rj = r + roff[j];
    const double s = sig[j];
    const float2* wj = w + (int64_t)j * n;
    const double2* dj = d + (int64_t)j * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 rv = rj[e], dv = dj[e];
        const float2 wv = wj[e];
        rj[e] = make_double2(rv.x - (double)wv.x + s * dv.x, rv.y - (double)wv.y + s * dv.y);
    }
}

// y_f = a_f + beta gamma5 s_f for nfield packed complex128 fields of vol sites: gamma5 =
// diag(1, 1, -1, -1) in spin negates spins 2 and 3, i.e. planes 3..5 of the packed
// field, its second half.
__global__ void k_gamma5_axpy(double2* __restrict__ y, const double2* __restrict__ a, const double2* __restrict__ sv,
                              double beta, int64_t half, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i % (2 * half);
        const double g = e < half ? beta : -beta;
        const double2 av = a[i], v = sv[i];
        y[i] = make_double2(av.x + g * v.x, av.y + g * v.y);
    }
}

inline unsigned grid_for(int64_t count) {
    int64_t g = (count + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

template <class T>
int reduce_blocks(int64_t n) {
    int64_t npk = n / Ops<T>::CPX;
    int64_t b = (npk + (int64_t)NT * PK - 1) / ((int64_t)NT * PK);
    return (int)(b < 1 ? 1 : b);
}

namespace {
int sm_count() {
    static const int n = [] {
        int d = 0, v = 0;
        if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
            v = 0;
        return v > 0 ? v : 152;
    }();
    return n;
}

// Packs per thread that nblk CTAs per column need for npk packs (0: too few CTAs).
int pk_for(int64_t npk, int nblk) {
    for (int pk = 1; pk <= 4; pk *= 2)
        if ((int64_t)NT * pk * nblk >= npk) return pk;
    return 0;
}
}  // namespace

// The vector kernels hold 4 CTAs of NT threads per SM (64 registers, 32 KB of
// shared memory).  A grid of 1.16 waves runs as long as 2 waves, so the CTAs per
// column are picked from PKT = 4, 2, 1 (in that order of preference) for a grid
// that fills at least 85 % of its last wave, else the fullest.
template <class T>
int wave_blocks(int64_t n, int ncol) {
    const int64_t npk = n / Ops<T>::CPX;
    const int64_t slots = (int64_t)sm_count() * 4;
    int best = 1;
    double best_eff = -1.0;
    for (int pk = 4; pk >= 1; pk /= 2) {
        int64_t nb = (npk + (int64_t)NT * pk - 1) / ((int64_t)NT * pk);
        if (nb < 1) nb = 1;
        const double waves = (double)(nb * (ncol > 0 ? ncol : 1)) / (double)slots;
        const double eff = waves / std::ceil(waves);
        if (eff >= 0.85) return (int)nb;
        if (eff > best_eff) {
            best_eff = eff;
            best = (int)nb;
        }
    }
    return best;
}

// Instantiate the kernel call for PKT = 1, 2 or 4.
#define SGN_PK_SWITCH(PKV, ...)               \
    switch (PKV) {                            \
        case 1: {                             \
            constexpr int PKT_ = 1;           \
            __VA_ARGS__;                      \
            break;                            \
        }                                     \
        case 2: {                             \
            constexpr int PKT_ = 2;           \
            __VA_ARGS__;                      \
            break;                            \
        }                                     \
        case 4: {                             \
            constexpr int PKT_ = 4;           \
            __VA_ARGS__;                      \
            break;                            \
        }                                     \
        default:                              \
            return cudaErrorInvalidValue;     \
    }

template <class T>
cudaError_t mdot(Basis<T> V, int J, const T* w, int64_t wsr, int64_t n, int ncol, const Reduce& rd, int with_norm,
                 const int* skip, cudaStream_t st) {
    if (J + 1 > MAXSLOT) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    dim3 grid(rd.nblk, ncol);
    SGN_PK_SWITCH(pk_for(npk, rd.nblk), k_mdot<T, PKT_><<<grid, NT, 0, st>>>(V, J, w, wsr, npk, rd, with_norm, skip))
    count_launch();
    return cudaGetLastError();
}

cudaError_t reduce(const Reduce& rd, int nslot, int ncol, int mode, int colidx, const DevState& S,
                   const double2* lambda, cudaStream_t st) {
    if (nslot > MAXSLOT) return cudaErrorInvalidValue;
    const int groups = (nslot + NWARP - 1) / NWARP;
    if (S.sums && S.rcount && groups > 1)
        k_reduce_split<<<dim3(ncol, groups), NT, 0, st>>>(rd, nslot, mode, colidx, S, lambda);
    else
        k_reduce<<<ncol, NT, 0, st>>>(rd, nslot, mode, colidx, S, lambda);
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t maxpy_mdot(Basis<T> V, int J, const double2* coef, int cstride, T* w, int64_t wsr, int64_t n, int ncol,
                       const Reduce& rd, const int* skip, cudaStream_t st) {
    if (J + 1 > MAXSLOT) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    dim3 grid(rd.nblk, ncol);
    SGN_PK_SWITCH(pk_for(npk, rd.nblk),
                  k_maxpy_mdot<T, PKT_><<<grid, NT, 0, st>>>(V, J, coef, cstride, w, wsr, npk, rd, skip))
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t maxpy_scale(Basis<T> V, int J, const double2* coef, int cstride, const T* w, int64_t wsr, T* out,
                        int64_t osr, const double* scale, int64_t n, int ncol, const int* skip, cudaStream_t st) {
    if (J > MAXSLOT) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    const int nb = wave_blocks<T>(n, ncol);
    dim3 grid(nb, ncol);
    SGN_PK_SWITCH(pk_for(npk, nb), k_maxpy_scale<T, PKT_><<<grid, NT, 0, st>>>(V, J, coef, cstride, w, wsr, out, osr,
                                                                              scale, npk, skip))
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t update_x(Basis<T> V, int J, const double2* coef, int cstride, double2* x, int64_t xsr, int64_t n,
                     int ncol, const int* skip, const int* kk, cudaStream_t st) {
    if (J > MAXSLOT) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    const int nb = wave_blocks<T>(n, ncol);
    dim3 grid(nb, ncol);
    SGN_PK_SWITCH(pk_for(npk, nb),
                  k_update_x<T, PKT_><<<grid, NT, 0, st>>>(V, J, coef, cstride, x, xsr, npk, skip, kk))
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t update_shifts(Basis<T> V, int J, const double2* y, int s, int kmax, double2* xs, int64_t xs_shift,
                          int64_t xs_col, int64_t n, int ncol, const int* skip, const int* kk, cudaStream_t st) {
    int64_t npk = n / Ops<T>::CPX;
    if (s <= 0 || npk <= 0) return cudaSuccess;
    // group size: SGN_SHIFT_GROUP = 1, 4, 8, 10 or 20 overrides the default 2 (measurements)
    static const int forced = [] {
        const char* e = getenv("SGN_SHIFT_GROUP");
        return e ? atoi(e) : 0;
    }();
    const int sg = (forced == 20 && s <= 20) || forced == 10 || forced == 8 || forced == 4 || forced == 1 ? forced : 2;
    size_t smem = sizeof(typename Ops<T>::C) * (size_t)(s < sg ? s : sg) * (size_t)J;
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    const int64_t tiles = (npk + NT - 1) / NT;
    const int64_t nblk = tiles * ((s + sg - 1) / sg);
    if (nblk > 0x7fffffff) return cudaErrorInvalidValue;
    dim3 grid((unsigned)nblk, ncol);
    if (sg == 20)
        k_update_shifts<T, 20><<<grid, NT, smem, st>>>(V, J, y, s, kmax, xs, xs_shift, xs_col, npk, skip, kk);
    else if (sg == 10)
        k_update_shifts<T, 10><<<grid, NT, smem, st>>>(V, J, y, s, kmax, xs, xs_shift, xs_col, npk, skip, kk);
    else if (sg == 8)
        k_update_shifts<T, 8><<<grid, NT, smem, st>>>(V, J, y, s, kmax, xs, xs_shift, xs_col, npk, skip, kk);
    else if (sg == 4)
        k_update_shifts<T, 4><<<grid, NT, smem, st>>>(V, J, y, s, kmax, xs, xs_shift, xs_col, npk, skip, kk);
    else if (sg == 1)
        k_update_shifts<T, 1><<<grid, NT, smem, st>>>(V, J, y, s, kmax, xs, xs_shift, xs_col, npk, skip, kk);
    else
        k_update_shifts<T, 2><<<grid, NT, smem, st>>>(V, J, y, s, kmax, xs, xs_shift, xs_col, npk, skip, kk);
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t dcgs_dots(Basis<T> V, int J, const T* u, const T* z, int64_t wsr, int64_t n, int ncol, const Reduce& rd,
                      const int* skip, cudaStream_t st) {
    if (2 * J + 3 > MAXSLOT) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    dim3 grid(rd.nblk, ncol);
    SGN_PK_SWITCH(pk_for(npk, rd.nblk), k_dcgs_dots<T, PKT_><<<grid, NT, 0, st>>>(V, J, u, z, wsr, npk, rd, skip))
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t dcgs_update(Basis<T> V, int J, const double2* coef, int cstride, T* u, const T* z, T* next, int64_t wsr,
                        int64_t n, int ncol, const int* skip, cudaStream_t st) {
    if (J > MAXSLOT) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    const int nb = wave_blocks<T>(n, ncol);
    dim3 grid(nb, ncol);
    SGN_PK_SWITCH(pk_for(npk, nb), k_dcgs_update<T, PKT_><<<grid, NT, 0, st>>>(V, J, coef, cstride, u, z, next, wsr,
                                                                              npk, skip))
    count_launch();
    return cudaGetLastError();
}

template cudaError_t dcgs_dots<double2>(Basis<double2>, int, const double2*, const double2*, int64_t, int64_t, int,
                                        const Reduce&, const int*, cudaStream_t);
template cudaError_t dcgs_dots<float2>(Basis<float2>, int, const float2*, const float2*, int64_t, int64_t, int,
                                       const Reduce&, const int*, cudaStream_t);
template cudaError_t dcgs_update<double2>(Basis<double2>, int, const double2*, int, double2*, const double2*,
                                          double2*, int64_t, int64_t, int, const int*, cudaStream_t);
template cudaError_t dcgs_update<float2>(Basis<float2>, int, const double2*, int, float2*, const float2*, float2*,
                                         int64_t, int64_t, int, const int*, cudaStream_t);

cudaError_t gamma5_axpy(double2* y, const double2* a, const double2* s, double beta, int64_t vol, int nfield,
                        cudaStream_t st) {
    const int64_t total = (int64_t)nfield * 12 * vol;
    if (total <= 0) return cudaSuccess;
    k_gamma5_axpy<<<grid_for(total), NT, 0, st>>>(y, a, s, beta, 6 * vol, total);
    count_launch();
    return cudaGetLastError();
}

cudaError_t correct_residuals(double2* r, const long long* roff, const double* sig, const float2* w,
                              const double2* d, int64_t n, int nb, cudaStream_t st) {
    if (nb < 1) return cudaSuccess;
    if (nb > 65535) return cudaErrorInvalidValue;
    unsigned gx = (unsigned)std::min<int64_t>((n + NT - 1) / NT, 1024);
    k_correct_residuals<<<dim3(gx, nb), NT, 0, st>>>(r, roff, sig, w, d, n);
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t axpby3(T* out, double a, const T* x, double b, const T* y, double c, const T* z, int64_t count,
                   cudaStream_t st) {
    int64_t npk = count / Ops<T>::CPX;
    k_axpby3<T><<<grid_for(npk), NT, 0, st>>>(out, a, x, b, y, c, z, npk);
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t block_combine(const T* Y, int q, const double2* Cm, int r, T* Z, int64_t n, cudaStream_t st) {
    if (q > MAXSLOT || r < 1) return cudaErrorInvalidValue;
    int64_t npk = n / Ops<T>::CPX;
    k_block_combine<T><<<(unsigned)((npk + NT - 1) / NT), NT, 0, st>>>(Y, q, Cm, r, Z, n, npk);
    count_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t random_fill(T* out, int64_t count, uint64_t seed, cudaStream_t st) {
    k_random_fill<T><<<grid_for(count), 256, 0, st>>>(out, count, seed);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t axpby3<double2>(double2*, double, const double2*, double, const double2*, double,
                                     const double2*, int64_t, cudaStream_t);
template cudaError_t axpby3<float2>(float2*, double, const float2*, double, const float2*, double, const float2*,
                                    int64_t, cudaStream_t);
template cudaError_t block_combine<double2>(const double2*, int, const double2*, int, double2*, int64_t,
                                            cudaStream_t);
template cudaError_t block_combine<float2>(const float2*, int, const double2*, int, float2*, int64_t, cudaStream_t);
template cudaError_t random_fill<double2>(double2*, int64_t, uint64_t, cudaStream_t);
template cudaError_t random_fill<float2>(float2*, int64_t, uint64_t, cudaStream_t);

cudaError_t convert_f64_to_f32(const double2* in, float2* out, int64_t count, cudaStream_t st) {
    k_f64_to_f32<<<grid_for(count), 256, 0, st>>>(in, out, count);
    count_launch();
    return cudaGetLastError();
}
cudaError_t convert_f32_to_f64(const float2* in, double2* out, int64_t count, cudaStream_t st) {
    k_f32_to_f64<<<grid_for(count), 256, 0, st>>>(in, out, count);
    count_launch();
    return cudaGetLastError();
}
cudaError_t links_f64_to_bf16(const double2* in, __nv_bfloat162* out, int64_t count, cudaStream_t st) {
    k_f64_to_bf16<<<grid_for(count), 256, 0, st>>>(in, out, count);
    count_launch();
    return cudaGetLastError();
}
cudaError_t links_f64_to_f16(const double2* in, __half2* out, int64_t count, cudaStream_t st) {
    k_f64_to_f16<<<grid_for(count), 256, 0, st>>>(in, out, count);
    count_launch();
    return cudaGetLastError();
}

#define SGN_INST(T)                                                                                              \
    template int reduce_blocks<T>(int64_t);                                                                      \
    template int wave_blocks<T>(int64_t, int);                                                                   \
    template cudaError_t mdot<T>(Basis<T>, int, const T*, int64_t, int64_t, int, const Reduce&, int, const int*, \
                                 cudaStream_t);                                                                  \
    template cudaError_t maxpy_mdot<T>(Basis<T>, int, const double2*, int, T*, int64_t, int64_t, int,           \
                                       const Reduce&, const int*, cudaStream_t);                                 \
    template cudaError_t maxpy_scale<T>(Basis<T>, int, const double2*, int, const T*, int64_t, T*, int64_t,     \
                                        const double*, int64_t, int, const int*, cudaStream_t);                  \
    template cudaError_t update_x<T>(Basis<T>, int, const double2*, int, double2*, int64_t, int64_t, int,       \
                                     const int*, const int*, cudaStream_t);                                      \
    template cudaError_t update_shifts<T>(Basis<T>, int, const double2*, int, int, double2*, int64_t, int64_t,  \
                                          int64_t, int, const int*, const int*, cudaStream_t);
SGN_INST(double2)
SGN_INST(float2)

}  // namespace sgn
