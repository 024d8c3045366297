// H_W(mu) = gamma5 D_W(mu) (Sec. 1 of the paper) in float-float arithmetic on the FP32 units:
// every real quantity is an unevaluated sum hi + lo of two floats (about 48 significant bits),
// the arithmetic built from error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA form of TwoProd) and, for the link products, a compensated dot product in the style of
// Ogita, Rump and Oishi's Dot2 (the sum and the product errors carried in a second float).
//
// Use: the mixed form's true residuals r_i = b~ - (A^2 - sigma_i) x_i need A^2 x_i to far better
// than FP32 (they decide convergence at 1e-8 ||b~||), and GB300 executes FP64 at 1/64 of its FP32
// rate: the FP64 stencil is bound by the FP64 pipe.  The float-float stencil reaches ~1e-13 of the
// FP64 result with FP32 instructions only.  Fields enter and leave as (hi, lo) pairs of packed FP32
// fields (the FP32 layout of stencil.cu); the links as float4 (U32, fl(U - U32)) per entry.  Same hop structure as stencil.cu: rank-2 spin projection, gamma5 folded into
// the store, one thread per site and field, CTA = SX sites x RB fields of one site tile.
#include "sgn_internal.cuh"

namespace sgn {
namespace {

struct ff {
    float hi, lo;
};

// Knuth's TwoSum: s + e = a + b exactly.  Explicit _rn intrinsics keep the compiler from
// contracting or reassociating the error terms.
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// Dekker's FastTwoSum (exact when |a| >= |b|).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// Sum of two float-float numbers, left unnormalised: hi is the rounded sum of the high parts, lo
// collects its error and the low parts (|lo| stays within a few units of 2^-24 |hi| unless the sum
// cancels, and hi + lo is the sum to about 2^-46 of the operands either way).  The stencil's
// intermediate sums and its accumulators use this form; the accumulators are normalised once,
// before the store.
__device__ __forceinline__ ff ff_add_u(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
// a * b: TwoProd of the high parts by FMA, the cross terms in FP32 (their rounding is of
// order 2^-48 of the product), the small lo * lo term dropped.
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// scaling by a float whose product is exact (a power of two: the hop coefficient -1/2 of the
// space directions)
__device__ __forceinline__ ff ff_scale2(ff a, float s) { return {a.hi * s, a.lo * s}; }

// Compensated dot-product accumulator: value s + c.  add(a, b) adds a * b: the product's
// rounding error (TwoProd) and the sum's (TwoSum) go into c.
struct Dot {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(ff a, ff b) {
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        const ff t = two_sum(s, p);
        s = t.hi;
        c = __fadd_rn(c, __fadd_rn(t.lo, e));
    }
    __device__ __forceinline__ ff value() const { return {s, c}; }  // unnormalised (see ff_add_u)
};

struct ffc {
    ff re, im;
};
__device__ __forceinline__ ffc cadd(ffc a, ffc b) { return {ff_add_u(a.re, b.re), ff_add_u(a.im, b.im)}; }
__device__ __forceinline__ ffc csub(ffc a, ffc b) { return {ff_add_u(a.re, ff_neg(b.re)), ff_add_u(a.im, ff_neg(b.im))}; }
__device__ __forceinline__ ffc mul_i(ffc a) { return {ff_neg(a.im), a.re}; }   // i a
__device__ __forceinline__ ffc mul_mi(ffc a) { return {a.im, ff_neg(a.re)}; }  // -i a

// 12 spin-colour entries of one site from the (hi, lo) packed fields: plane p holds entries
// 2p, 2p + 1 at float2 offset p * 2 vol + 2 site.
__device__ __forceinline__ void load_site(const float2* __restrict__ fh, const float2* __restrict__ fl, int64_t site,
                                          int64_t vol2, ffc (&p)[12]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 h = __ldg(reinterpret_cast<const float4*>(fh + k * vol2 + 2 * site));
        const float4 l = __ldg(reinterpret_cast<const float4*>(fl + k * vol2 + 2 * site));
        p[2 * k] = {{h.x, l.x}, {h.y, l.y}};
        p[2 * k + 1] = {{h.z, l.z}, {h.w, l.w}};
    }
}

// Spin projection h = psi_up + S B psi_dn (B = -i sigma_{x,y,z}, or 1 for t; see stencil.cu).
template <int NU, int S>
__device__ __forceinline__ void project(const ffc (&p)[12], ffc (&h0)[3], ffc (&h1)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const ffc p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if constexpr (NU == 0) {  // (-i p3, -i p2)
            h0[c] = S > 0 ? cadd(p0, mul_mi(p3)) : csub(p0, mul_mi(p3));
            h1[c] = S > 0 ? cadd(p1, mul_mi(p2)) : csub(p1, mul_mi(p2));
        } else if constexpr (NU == 1) {  // (-p3, p2)
            h0[c] = S > 0 ? csub(p0, p3) : cadd(p0, p3);
            h1[c] = S > 0 ? cadd(p1, p2) : csub(p1, p2);
        } else if constexpr (NU == 2) {  // (-i p2, i p3)
            h0[c] = S > 0 ? cadd(p0, mul_mi(p2)) : csub(p0, mul_mi(p2));
            h1[c] = S > 0 ? cadd(p1, mul_i(p3)) : csub(p1, mul_i(p3));
        } else {  // (p2, p3)
            h0[c] = S > 0 ? cadd(p0, p2) : csub(p0, p2);
            h1[c] = S > 0 ? cadd(p1, p3) : csub(p1, p3);
        }
    }
}

// acc += coef (1 + S gamma_NU) W psi(nb), W = U_NU(site) (S = -1) or U_NU(nb)^dag (S = +1).
// coef: -1/2 (times -1 across an antiperiodic boundary) in the space directions, applied
// exactly; -1/2 e^{+-mu} in time, a float-float product.
template <int NU, int S>
__device__ __forceinline__ void hop(ffc (&acc)[12], const float2* __restrict__ fh, const float2* __restrict__ fl,
                                    const float4* __restrict__ Uf, int64_t link_site,
                                    int64_t nb, ff coef, int64_t vol) {
    ffc h0[3], h1[3];
    {
        ffc p[12];
        load_site(fh, fl, nb, 2 * vol, p);
        project<NU, S>(p, h0, h1);
    }
    const int64_t lb = (int64_t)NU * 9 * vol + link_site;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Dot g0r, g0i, g1r, g1i;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int64_t e = lb + (int64_t)(S < 0 ? a * 3 + b : b * 3 + a) * vol;
            const float4 u = __ldg(Uf + e);  // (Re hi, Im hi, Re lo, Im lo)
            const ff ur = {u.x, u.z};
            // U h (forward) or conj(U) h (backward, the dagger's transpose is in the index)
            const ff ui = S < 0 ? ff{u.y, u.w} : ff{-u.y, -u.w};
            const ff nui = ff_neg(ui);
            g0r.add(ur, h0[b].re);
            g0r.add(nui, h0[b].im);
            g0i.add(ur, h0[b].im);
            g0i.add(ui, h0[b].re);
            g1r.add(ur, h1[b].re);
            g1r.add(nui, h1[b].im);
            g1i.add(ur, h1[b].im);
            g1i.add(ui, h1[b].re);
        }
        ffc g0 = {g0r.value(), g0i.value()}, g1 = {g1r.value(), g1i.value()};
        if (NU == 3 || coef.lo != 0.f) {  // the space directions' -1/2 is exact: lo = 0
            g0 = {ff_mul(g0.re, coef), ff_mul(g0.im, coef)};
            g1 = {ff_mul(g1.re, coef), ff_mul(g1.im, coef)};
        } else {
            g0 = {ff_scale2(g0.re, coef.hi), ff_scale2(g0.im, coef.hi)};
            g1 = {ff_scale2(g1.re, coef.hi), ff_scale2(g1.im, coef.hi)};
        }
        acc[a] = cadd(acc[a], g0);
        acc[3 + a] = cadd(acc[3 + a], g1);
        // lower spins: S B^dag g
        if constexpr (NU == 0) {  // B^dag g = (i g1, i g0)
            acc[6 + a] = S > 0 ? cadd(acc[6 + a], mul_i(g1)) : csub(acc[6 + a], mul_i(g1));
            acc[9 + a] = S > 0 ? cadd(acc[9 + a], mul_i(g0)) : csub(acc[9 + a], mul_i(g0));
        } else if constexpr (NU == 1) {  // (g1, -g0)
            acc[6 + a] = S > 0 ? cadd(acc[6 + a], g1) : csub(acc[6 + a], g1);
            acc[9 + a] = S > 0 ? csub(acc[9 + a], g0) : cadd(acc[9 + a], g0);
        } else if constexpr (NU == 2) {  // (i g0, -i g1)
            acc[6 + a] = S > 0 ? cadd(acc[6 + a], mul_i(g0)) : csub(acc[6 + a], mul_i(g0));
            acc[9 + a] = S > 0 ? cadd(acc[9 + a], mul_mi(g1)) : csub(acc[9 + a], mul_mi(g1));
        } else {  // (g0, g1)
            acc[6 + a] = S > 0 ? cadd(acc[6 + a], g0) : csub(acc[6 + a], g0);
            acc[9 + a] = S > 0 ? cadd(acc[9 + a], g1) : csub(acc[9 + a], g1);
        }
    }
}

__device__ __forceinline__ ff coef_ff(float hi, float lo, bool flip) { return flip ? ff{-hi, -lo} : ff{hi, lo}; }

template <int NU>
__device__ __forceinline__ void both_hops(ffc (&acc)[12], const float2* __restrict__ fh, const float2* __restrict__ fl,
                                          const float4* __restrict__ Uf, int64_t site,
                                          const int co[4], const StencilParams& P) {
    int64_t stride = 1;
#pragma unroll
    for (int d = 0; d < NU; ++d) stride *= P.L[d];
    const int L = P.L[NU];
    int64_t fw = site + stride;
    bool ffl = false;
    if (co[NU] == L - 1) {
        fw = site - (int64_t)(L - 1) * stride;
        ffl = P.ap[NU];
    }
    int64_t bw = site - stride;
    bool bfl = false;
    if (co[NU] == 0) {
        bw = site + (int64_t)(L - 1) * stride;
        bfl = P.ap[NU];
    }
    hop<NU, -1>(acc, fh, fl, Uf, site, fw, coef_ff(P.cf32[NU], P.cf_lo[NU], ffl), P.vol);
    hop<NU, +1>(acc, fh, fl, Uf, bw, bw, coef_ff(P.cb32[NU], P.cb_lo[NU], bfl), P.vol);
}

// Thread (x, y) of CTA b: site (b / ngrp) * SX + x, field (b % ngrp) * RB + y.  Capped at 128
// registers (four CTAs of 128 threads per SM; as the compiler sizes it, 144 registers and three
// CTAs ran 20 % slower at 10^4 despite a few spilled values).
__global__ void __launch_bounds__(128, 4)
    k_hw_ff(float2* __restrict__ oh, float2* __restrict__ ol, const float2* __restrict__ ih,
            const float2* __restrict__ il, const float4* __restrict__ Uf, int nrhs,
            StencilParams P, int ngrp) {
    const int64_t tile = blockIdx.x / (unsigned)ngrp;
    const int grp = (int)(blockIdx.x - tile * ngrp);
    const int64_t site = tile * blockDim.x + threadIdx.x;
    const int rhs = grp * blockDim.y + threadIdx.y;
    if (site >= P.vol || rhs >= nrhs) return;
    const float2* fh = ih + rhs * P.stride_rhs;
    const float2* fl = il + rhs * P.stride_rhs;
    int co[4];
    {
        const uint32_t s0 = (uint32_t)site;
        const uint32_t q0 = P.div[0].div(s0);
        co[0] = (int)(s0 - q0 * (uint32_t)P.L[0]);
        const uint32_t q1 = P.div[1].div(q0);
        co[1] = (int)(q0 - q1 * (uint32_t)P.L[1]);
        const uint32_t q2 = P.div[2].div(q1);
        co[2] = (int)(q1 - q2 * (uint32_t)P.L[2]);
        co[3] = (int)q2;
    }
    ffc acc[12];
    {
        load_site(fh, fl, site, 2 * P.vol, acc);
        const ff d = {P.diag32, P.diag_lo};
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {ff_mul(acc[k].re, d), ff_mul(acc[k].im, d)};
    }
    both_hops<0>(acc, fh, fl, Uf, site, co, P);
    both_hops<1>(acc, fh, fl, Uf, site, co, P);
    both_hops<2>(acc, fh, fl, Uf, site, co, P);
    both_hops<3>(acc, fh, fl, Uf, site, co, P);
    float2* gh = oh + rhs * P.stride_rhs;
    float2* gl = ol + rhs * P.stride_rhs;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float g = k < 3 ? 1.f : -1.f;  // gamma5 = diag(1, 1, -1, -1): planes 3..5 hold spins 2, 3
        const ff ar = two_sum(acc[2 * k].re.hi, acc[2 * k].re.lo), ai = two_sum(acc[2 * k].im.hi, acc[2 * k].im.lo);
        const ff br = two_sum(acc[2 * k + 1].re.hi, acc[2 * k + 1].re.lo),
                 bi = two_sum(acc[2 * k + 1].im.hi, acc[2 * k + 1].im.lo);
        const ffc a = {ar, ai}, b = {br, bi};
        *reinterpret_cast<float4*>(gh + k * 2 * P.vol + 2 * site) =
            make_float4(g * a.re.hi, g * a.im.hi, g * b.re.hi, g * b.im.hi);
        *reinterpret_cast<float4*>(gl + k * 2 * P.vol + 2 * site) =
            make_float4(g * a.re.lo, g * a.im.lo, g * b.re.lo, g * b.im.lo);
    }
}

// hi = fl(v), lo = fl(v - hi): v = hi + lo to about 2^-48 relative.
__global__ void k_split_ff(const double2* __restrict__ in, float2* __restrict__ hi, float2* __restrict__ lo,
                           int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = in[i];
        const float hx = (float)v.x, hy = (float)v.y;
        hi[i] = make_float2(hx, hy);
        lo[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
}
// out = hi + lo in FP64
__global__ void k_join_ff(const float2* __restrict__ hi, const float2* __restrict__ lo, double2* __restrict__ out,
                          int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 h = hi[i], l = lo[i];
        out[i] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
}
// r = b - (yh + yl) + sigma x, FP64 (the true residual of (A^2 - sigma) x = b with y = A^2 x)
__global__ void k_residual_ff(double2* __restrict__ r, const double2* __restrict__ b, const float2* __restrict__ yh,
                              const float2* __restrict__ yl, double sigma, const double2* __restrict__ x,
                              int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 h = yh[i], l = yl[i];
        const double2 bv = b[i], xv = x[i];
        r[i] = make_double2(bv.x - ((double)h.x + (double)l.x) + sigma * xv.x,
                            bv.y - ((double)h.y + (double)l.y) + sigma * xv.y);
    }
}
// links as float-float pairs, one 16-byte load per entry: (Re hi, Im hi, Re lo, Im lo) with
// hi = U32 and lo = fl(U - U32)
__global__ void k_links_ff(const double2* __restrict__ U, const float2* __restrict__ U32, float4* __restrict__ out,
                           int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 u = U[i];
        const float2 h = U32[i];
        out[i] = make_float4(h.x, h.y, (float)(u.x - (double)h.x), (float)(u.y - (double)h.y));
    }
}

unsigned grid_of(int64_t count) {
    const int64_t b = (count + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_hw_ff(float2* oh, float2* ol, const float2* ih, const float2* il, const float4* Uf, int nrhs,
                         const StencilParams& p, cudaStream_t st) {
    if (nrhs <= 0 || p.vol <= 0) return cudaSuccess;
    // 64 sites x 2 fields per CTA (128 x 1 for one field); the fields of a site tile in
    // consecutive CTAs share links in L2
    const int rb = nrhs >= 2 ? 2 : 1, sx = 128 / rb;
    const int ngrp = (nrhs + rb - 1) / rb;
    const int64_t tiles = (p.vol + sx - 1) / sx;
    if (tiles * ngrp > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_hw_ff<<<(unsigned)(tiles * ngrp), dim3(sx, rb), 0, st>>>(oh, ol, ih, il, Uf, nrhs, p, ngrp);
    count_launch();
    return cudaGetLastError();
}

cudaError_t split_ff(const double2* in, float2* hi, float2* lo, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_split_ff<<<grid_of(count), 256, 0, st>>>(in, hi, lo, count);
    count_launch();
    return cudaGetLastError();
}
cudaError_t join_ff(const float2* hi, const float2* lo, double2* out, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_join_ff<<<grid_of(count), 256, 0, st>>>(hi, lo, out, count);
    count_launch();
    return cudaGetLastError();
}
cudaError_t residual_ff(double2* r, const double2* b, const float2* yh, const float2* yl, double sigma,
                        const double2* x, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_residual_ff<<<grid_of(count), 256, 0, st>>>(r, b, yh, yl, sigma, x, count);
    count_launch();
    return cudaGetLastError();
}
cudaError_t links_ff(const double2* U, const float2* U32, float4* out, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_links_ff<<<grid_of(count), 256, 0, st>>>(U, U32, out, count);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sgn
