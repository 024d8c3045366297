// Wilson kernel H_W(mu) = gamma5 D_W(mu) on nrhs fields (Sec. 1 of the paper;
// D_W(mu) with e^{+mu} on forward and e^{-mu} on backward time hops).
//
// One thread computes one site of one field.  A CTA covers SX consecutive
// sites (x fastest) for RB fields, so the RB warps that share a site tile
// read the same links back to back and the link bytes come from L1 after the
// first field: with 12 fields the links cost 1/12 of their bytes per field.
// Fields and links are in the packed layout (planes over sites), so every
// load of a warp covers 32 consecutive sites of one plane.
// Each hop uses the rank-2 spin projector (1 -/+ gamma_nu): two colour
// vectors are multiplied by the link instead of four, and gamma5 is folded
// into the write (spins 2, 3 negated).
#include "sgn_internal.cuh"

namespace sgn {
namespace {

template <class R>
struct Cx {
    R x, y;
};
template <class R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) { return {-a.y, a.x}; }   // i a
template <class R>
__device__ __forceinline__ Cx<R> mul_mi(Cx<R> a) { return {a.y, -a.x}; }  // -i a
template <class R>
__device__ __forceinline__ Cx<R> scale(Cx<R> a, R s) { return {a.x * s, a.y * s}; }
// acc += u * v
template <class R>
__device__ __forceinline__ void cmac(Cx<R>& acc, Cx<R> u, Cx<R> v) {
    acc.x = fma(u.x, v.x, acc.x);
    acc.x = fma(-u.y, v.y, acc.x);
    acc.y = fma(u.x, v.y, acc.y);
    acc.y = fma(u.y, v.x, acc.y);
}
// acc += conj(u) * v
template <class R>
__device__ __forceinline__ void cmac_conj(Cx<R>& acc, Cx<R> u, Cx<R> v) {
    acc.x = fma(u.x, v.x, acc.x);
    acc.x = fma(u.y, v.y, acc.x);
    acc.y = fma(u.x, v.y, acc.y);
    acc.y = fma(-u.y, v.x, acc.y);
}

// ---- loads -----------------------------------------------------------------
// Packed field: plane p (entries 2p, 2p+1) of site s at complex offset p * vol2 + 2 s.
template <class R>
struct Field;
template <>
struct Field<double> {
    using T = double2;
    static __device__ __forceinline__ void load(const double2* __restrict__ f, int64_t site, int64_t vol2,
                                                Cx<double> p[12]) {
        const double2* s = f + 2 * site;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 a = __ldg(s + k * vol2);
            const double2 b = __ldg(s + k * vol2 + 1);
            p[2 * k] = {a.x, a.y};
            p[2 * k + 1] = {b.x, b.y};
        }
    }
    // CS: evict-first stores (see k_hw)
    template <bool CS>
    static __device__ __forceinline__ void store(double2* __restrict__ f, int64_t site, int64_t vol2,
                                                 const Cx<double> p[12]) {
        double2* s = f + 2 * site;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 a = make_double2(p[2 * k].x, p[2 * k].y), b = make_double2(p[2 * k + 1].x, p[2 * k + 1].y);
            if constexpr (CS) {
                __stcs(s + k * vol2, a);
                __stcs(s + k * vol2 + 1, b);
            } else {
                s[k * vol2] = a;
                s[k * vol2 + 1] = b;
            }
        }
    }
};
template <>
struct Field<float> {
    using T = float2;
    static __device__ __forceinline__ void load(const float2* __restrict__ f, int64_t site, int64_t vol2,
                                                Cx<float> p[12]) {
        const float2* s = f + 2 * site;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(s + k * vol2));
            p[2 * k] = {v.x, v.y};
            p[2 * k + 1] = {v.z, v.w};
        }
    }
    template <bool CS>
    static __device__ __forceinline__ void store(float2* __restrict__ f, int64_t site, int64_t vol2,
                                                 const Cx<float> p[12]) {
        float2* s = f + 2 * site;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = make_float4(p[2 * k].x, p[2 * k].y, p[2 * k + 1].x, p[2 * k + 1].y);
            if constexpr (CS)
                __stcs(reinterpret_cast<float4*>(s + k * vol2), v);
            else
                *reinterpret_cast<float4*>(s + k * vol2) = v;
        }
    }
};

template <class R, class LinkT>
struct Link;
template <>
struct Link<double, double2> {
    static __device__ __forceinline__ Cx<double> ld(const double2* __restrict__ U, int64_t i) {
        double2 v = __ldg(U + i);
        return {v.x, v.y};
    }
};
template <>
struct Link<float, float2> {
    static __device__ __forceinline__ Cx<float> ld(const float2* __restrict__ U, int64_t i) {
        float2 v = __ldg(U + i);
        return {v.x, v.y};
    }
};
template <>
struct Link<float, __nv_bfloat162> {
    static __device__ __forceinline__ Cx<float> ld(const __nv_bfloat162* __restrict__ U, int64_t i) {
        float2 v = __bfloat1622float2(U[i]);
        return {v.x, v.y};
    }
};
template <>
struct Link<float, __half2> {
    static __device__ __forceinline__ Cx<float> ld(const __half2* __restrict__ U, int64_t i) {
        float2 v = __half22float2(__ldg(U + i));
        return {v.x, v.y};
    }
};

// One hop for NR fields: acc[i] += coef * (1 + S gamma_NU) W psi_i(nb), W =
// U_NU(site) (forward, S = -1) or U_NU(nb)^dag (backward, S = +1).  Spin
// index a*3 + colour c.
//   (1 + S gamma) psi = [h ; S B^dag h],  h = psi_up + S B psi_dn,
//   gamma_NU = [[0, B], [B^dag, 0]]:  B = -i sigma_{x,y,z}, or 1 for t.
// Each link entry is loaded once and applied to the NR fields.

// Spin projection h = psi_up + S B psi_dn of one neighbour spinor.
template <class R, int NU, int S>
__device__ __forceinline__ void project(const Cx<R> (&p)[12], Cx<R> (&h0)[3], Cx<R> (&h1)[3]) {
    const R s = R(S);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Cx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if constexpr (NU == 0) {  // B psi_dn = (-i p3, -i p2)
            h0[c] = p0 + scale(mul_mi(p3), s);
            h1[c] = p1 + scale(mul_mi(p2), s);
        } else if constexpr (NU == 1) {  // (-p3, p2)
            h0[c] = p0 - scale(p3, s);
            h1[c] = p1 + scale(p2, s);
        } else if constexpr (NU == 2) {  // (-i p2, i p3)
            h0[c] = p0 + scale(mul_mi(p2), s);
            h1[c] = p1 + scale(mul_i(p3), s);
        } else {  // (p2, p3)
            h0[c] = p0 + scale(p2, s);
            h1[c] = p1 + scale(p3, s);
        }
    }
}

// The link multiplication and the reconstruction into acc for NR projected spinors.
template <class R, class LinkT, int NU, int S, int NR>
__device__ __forceinline__ void hop_links(Cx<R> (&acc)[NR][12], const Cx<R> (&h0)[NR][3], const Cx<R> (&h1)[NR][3],
                                          const LinkT* __restrict__ U, int64_t link_site, R coef, int64_t vol) {
    const R s = R(S);
    // packed links: entry (row, col) of U_NU(site) at ((NU * 9 + 3 row + col) * vol + site)
    const LinkT* lb = U + (int64_t)NU * 9 * vol + link_site;
    const R cs = coef * s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Cx<R> g0[NR], g1[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            g0[i] = {R(0), R(0)};
            g1[i] = {R(0), R(0)};
        }
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if constexpr (S < 0) {  // U(site) h
                const Cx<R> u = Link<R, LinkT>::ld(lb, (a * 3 + b) * vol);
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    cmac(g0[i], u, h0[i][b]);
                    cmac(g1[i], u, h1[i][b]);
                }
            } else {  // U(nb)^dag h: (U^dag)_{ab} = conj(U_{ba})
                const Cx<R> u = Link<R, LinkT>::ld(lb, (b * 3 + a) * vol);
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    cmac_conj(g0[i], u, h0[i][b]);
                    cmac_conj(g1[i], u, h1[i][b]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            acc[i][a] = acc[i][a] + scale(g0[i], coef);
            acc[i][3 + a] = acc[i][3 + a] + scale(g1[i], coef);
            if constexpr (NU == 0) {  // B^dag g = (i g1, i g0)
                acc[i][6 + a] = acc[i][6 + a] + scale(mul_i(g1[i]), cs);
                acc[i][9 + a] = acc[i][9 + a] + scale(mul_i(g0[i]), cs);
            } else if constexpr (NU == 1) {  // (g1, -g0)
                acc[i][6 + a] = acc[i][6 + a] + scale(g1[i], cs);
                acc[i][9 + a] = acc[i][9 + a] - scale(g0[i], cs);
            } else if constexpr (NU == 2) {  // (i g0, -i g1)
                acc[i][6 + a] = acc[i][6 + a] + scale(mul_i(g0[i]), cs);
                acc[i][9 + a] = acc[i][9 + a] + scale(mul_mi(g1[i]), cs);
            } else {  // (g0, g1)
                acc[i][6 + a] = acc[i][6 + a] + scale(g0[i], cs);
                acc[i][9 + a] = acc[i][9 + a] + scale(g1[i], cs);
            }
        }
    }
}


template <class R, class LinkT, int NU, int S, int NR>
__device__ __forceinline__ void hop(Cx<R> (&acc)[NR][12], const typename Field<R>::T* __restrict__ in,
                                    int64_t stride_rhs, const bool (&act)[NR], const LinkT* __restrict__ U,
                                    int64_t link_site, int64_t nb, R coef, int64_t vol) {
    Cx<R> h0[NR][3], h1[NR][3];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        Cx<R> p[12];
        if (act[i]) {
            Field<R>::load(in + i * stride_rhs, nb, 2 * vol, p);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) p[k] = {R(0), R(0)};
        }
        project<R, NU, S>(p, h0[i], h1[i]);
    }
    hop_links<R, LinkT, NU, S, NR>(acc, h0, h1, U, link_site, coef, vol);
}

template <class R>
__device__ __forceinline__ R cf_of(const StencilParams& P, int nu) {
    if constexpr (sizeof(R) == 4) return P.cf32[nu]; else return P.cf[nu];
}
template <class R>
__device__ __forceinline__ R cb_of(const StencilParams& P, int nu) {
    if constexpr (sizeof(R) == 4) return P.cb32[nu]; else return P.cb[nu];
}
template <class R>
__device__ __forceinline__ R diag_of(const StencilParams& P) {
    if constexpr (sizeof(R) == 4) return P.diag32; else return P.diag;
}

template <class R, class LinkT, int NU, int NR>
__device__ __forceinline__ void both_hops(Cx<R> (&acc)[NR][12], const typename Field<R>::T* __restrict__ in,
                                          const bool (&act)[NR], const LinkT* __restrict__ U, int64_t site,
                                          const int co[4], const StencilParams& P) {
    int64_t stride = 1;
#pragma unroll
    for (int d = 0; d < NU; ++d) stride *= P.L[d];
    const int L = P.L[NU];
    // forward neighbour
    int64_t fw = site + stride;
    R cf = cf_of<R>(P, NU);
    if (co[NU] == L - 1) {
        fw = site - (int64_t)(L - 1) * stride;
        if (P.ap[NU]) cf = -cf;
    }
    int64_t bw = site - stride;
    R cb = cb_of<R>(P, NU);
    if (co[NU] == 0) {
        bw = site + (int64_t)(L - 1) * stride;
        if (P.ap[NU]) cb = -cb;
    }
    hop<R, LinkT, NU, -1, NR>(acc, in, P.stride_rhs, act, U, site, fw, cf, P.vol);
    hop<R, LinkT, NU, +1, NR>(acc, in, P.stride_rhs, act, U, bw, bw, cb, P.vol);
}

// CTA b of the 1D grid covers site tile b / ngrp and field group b % ngrp: the
// field groups of a site tile run back to back, so the link and neighbour lines
// they share are read from HBM once (with the tile index fastest, each field
// group would sweep the whole lattice and re-read every link from HBM).
// Thread (x, y): site tile * SX + x, fields NR (group * RB + y) + 0..NR-1.
// CS: evict-first stores, for field sets far larger than L2, where a spinor is
// last read as the neighbour of a site one time slice away and the streaming
// result would otherwise push it out of L2 first.
template <class R, class LinkT, int NR, bool CS>
__global__ void __launch_bounds__(NR == 1 ? 384 : 256)
    k_hw(typename Field<R>::T* __restrict__ out, const typename Field<R>::T* __restrict__ in,
         const LinkT* __restrict__ U, int nrhs, StencilParams P, const int* __restrict__ skip, int ngrp) {
    const int64_t tile = blockIdx.x / (unsigned)ngrp;
    const int grp = (int)(blockIdx.x - tile * ngrp);
    const int64_t site = tile * blockDim.x + threadIdx.x;
    const int rhs0 = (grp * blockDim.y + threadIdx.y) * NR;
    if (site >= P.vol || rhs0 >= nrhs) return;
    bool act[NR];
    bool any = false;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        act[i] = rhs0 + i < nrhs && !(skip && skip[rhs0 + i]);
        any |= act[i];
    }
    if (!any) return;
    const typename Field<R>::T* fin = in + rhs0 * P.stride_rhs;
    int co[4];
    {
        // coordinates by exact multiply-shift division (no 64-bit integer division)
        const uint32_t s0 = (uint32_t)site;
        const uint32_t q0 = P.div[0].div(s0);
        co[0] = (int)(s0 - q0 * (uint32_t)P.L[0]);
        const uint32_t q1 = P.div[1].div(q0);
        co[1] = (int)(q0 - q1 * (uint32_t)P.L[1]);
        const uint32_t q2 = P.div[2].div(q1);
        co[2] = (int)(q1 - q2 * (uint32_t)P.L[2]);
        co[3] = (int)q2;
    }
    Cx<R> acc[NR][12];
    const R d = diag_of<R>(P);
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        if (act[i]) {
            Field<R>::load(fin + i * P.stride_rhs, site, 2 * P.vol, acc[i]);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[i][k] = {R(0), R(0)};
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[i][k] = scale(acc[i][k], d);
    }
    both_hops<R, LinkT, 0, NR>(acc, fin, act, U, site, co, P);
    both_hops<R, LinkT, 1, NR>(acc, fin, act, U, site, co, P);
    both_hops<R, LinkT, 2, NR>(acc, fin, act, U, site, co, P);
    both_hops<R, LinkT, 3, NR>(acc, fin, act, U, site, co, P);
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        if (!act[i]) continue;
        // gamma5 = diag(1, 1, -1, -1)
#pragma unroll
        for (int k = 6; k < 12; ++k) acc[i][k] = {-acc[i][k].x, -acc[i][k].y};
        Field<R>::template store<CS>(out + (rhs0 + i) * P.stride_rhs, site, 2 * P.vol, acc[i]);
    }
}

// ---- paired FP32 form --------------------------------------------------------
// Two fields per thread with their arithmetic paired: every real quantity is a
// float2 (field 0, field 1), so one packed FP32 instruction (FFMA2 on sm_100 and
// later) does the work of two.  The link entries are the same for both fields,
// so each complex multiply-add of the link products and the reconstruction is two
// paired FMAs instead of four scalar ones.  The spin projection stays scalar per
// field (its results land in the halves of the pairs).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <class LinkT, int NU, int S>
__device__ __forceinline__ void hop_x2(float2 (&ar)[12], float2 (&ai)[12], const float2* __restrict__ in,
                                       int64_t stride_rhs, const bool (&act)[2], const LinkT* __restrict__ U,
                                       int64_t link_site, int64_t nb, float coef, int64_t vol) {
    float2 hr0[3], hi0[3], hr1[3], hi1[3];  // the two projected colour vectors, paired over fields
    {
        Cx<float> pa[12], pb[12], ha0[3], ha1[3], hb0[3], hb1[3];
        if (act[0]) {
            Field<float>::load(in, nb, 2 * vol, pa);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) pa[k] = {0.f, 0.f};
        }
        if (act[1]) {
            Field<float>::load(in + stride_rhs, nb, 2 * vol, pb);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) pb[k] = {0.f, 0.f};
        }
        project<float, NU, S>(pa, ha0, ha1);
        project<float, NU, S>(pb, hb0, hb1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            hr0[c] = f2(ha0[c].x, hb0[c].x);
            hi0[c] = f2(ha0[c].y, hb0[c].y);
            hr1[c] = f2(ha1[c].x, hb1[c].x);
            hi1[c] = f2(ha1[c].y, hb1[c].y);
        }
    }
    const LinkT* lb = U + (int64_t)NU * 9 * vol + link_site;
    const float2 cc = f2s(coef), cs = f2s(coef * float(S)), ncs = f2s(-coef * float(S));
    // the sign of the Im u terms goes on the three projected pairs it multiplies (six negated
    // pairs per hop) instead of on a third broadcast pair per link entry (nine per hop)
    float2 n0[3], n1[3];  // -hi (g += u h) or -hr (g += conj(u) h)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        n0[b] = S < 0 ? f2(-hi0[b].x, -hi0[b].y) : f2(-hr0[b].x, -hr0[b].y);
        n1[b] = S < 0 ? f2(-hi1[b].x, -hi1[b].y) : f2(-hr1[b].x, -hr1[b].y);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 g0r = f2s(0.f), g0i = f2s(0.f), g1r = f2s(0.f), g1i = f2s(0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const Cx<float> u = Link<float, LinkT>::ld(lb, (S < 0 ? a * 3 + b : b * 3 + a) * vol);
            const float2 ux = f2s(u.x), uy = f2s(u.y);
            if constexpr (S < 0) {  // g += u h
                g0r = pfma(ux, hr0[b], g0r);
                g0r = pfma(uy, n0[b], g0r);
                g0i = pfma(ux, hi0[b], g0i);
                g0i = pfma(uy, hr0[b], g0i);
                g1r = pfma(ux, hr1[b], g1r);
                g1r = pfma(uy, n1[b], g1r);
                g1i = pfma(ux, hi1[b], g1i);
                g1i = pfma(uy, hr1[b], g1i);
            } else {  // g += conj(u) h
                g0r = pfma(ux, hr0[b], g0r);
                g0r = pfma(uy, hi0[b], g0r);
                g0i = pfma(ux, hi0[b], g0i);
                g0i = pfma(uy, n0[b], g0i);
                g1r = pfma(ux, hr1[b], g1r);
                g1r = pfma(uy, hi1[b], g1r);
                g1i = pfma(ux, hi1[b], g1i);
                g1i = pfma(uy, n1[b], g1i);
            }
        }
        ar[a] = pfma(cc, g0r, ar[a]);
        ai[a] = pfma(cc, g0i, ai[a]);
        ar[3 + a] = pfma(cc, g1r, ar[3 + a]);
        ai[3 + a] = pfma(cc, g1i, ai[3 + a]);
        if constexpr (NU == 0) {  // lower = (i g1, i g0) cs
            ar[6 + a] = pfma(ncs, g1i, ar[6 + a]);
            ai[6 + a] = pfma(cs, g1r, ai[6 + a]);
            ar[9 + a] = pfma(ncs, g0i, ar[9 + a]);
            ai[9 + a] = pfma(cs, g0r, ai[9 + a]);
        } else if constexpr (NU == 1) {  // (g1, -g0) cs
            ar[6 + a] = pfma(cs, g1r, ar[6 + a]);
            ai[6 + a] = pfma(cs, g1i, ai[6 + a]);
            ar[9 + a] = pfma(ncs, g0r, ar[9 + a]);
            ai[9 + a] = pfma(ncs, g0i, ai[9 + a]);
        } else if constexpr (NU == 2) {  // (i g0, -i g1) cs
            ar[6 + a] = pfma(ncs, g0i, ar[6 + a]);
            ai[6 + a] = pfma(cs, g0r, ai[6 + a]);
            ar[9 + a] = pfma(cs, g1i, ar[9 + a]);
            ai[9 + a] = pfma(ncs, g1r, ai[9 + a]);
        } else {  // (g0, g1) cs
            ar[6 + a] = pfma(cs, g0r, ar[6 + a]);
            ai[6 + a] = pfma(cs, g0i, ai[6 + a]);
            ar[9 + a] = pfma(cs, g1r, ar[9 + a]);
            ai[9 + a] = pfma(cs, g1i, ai[9 + a]);
        }
    }
}

template <class LinkT, int NU>
__device__ __forceinline__ void both_hops_x2(float2 (&ar)[12], float2 (&ai)[12], const float2* __restrict__ in,
                                             const bool (&act)[2], const LinkT* __restrict__ U, int64_t site,
                                             const int co[4], const StencilParams& P) {
    int64_t stride = 1;
#pragma unroll
    for (int d = 0; d < NU; ++d) stride *= P.L[d];
    const int L = P.L[NU];
    int64_t fw = site + stride;
    float cf = P.cf32[NU];
    if (co[NU] == L - 1) {
        fw = site - (int64_t)(L - 1) * stride;
        if (P.ap[NU]) cf = -cf;
    }
    int64_t bw = site - stride;
    float cb = P.cb32[NU];
    if (co[NU] == 0) {
        bw = site + (int64_t)(L - 1) * stride;
        if (P.ap[NU]) cb = -cb;
    }
    hop_x2<LinkT, NU, -1>(ar, ai, in, P.stride_rhs, act, U, site, fw, cf, P.vol);
    hop_x2<LinkT, NU, +1>(ar, ai, in, P.stride_rhs, act, U, bw, bw, cb, P.vol);
}

// One site, fields rhs0 and rhs0 + 1.
template <class LinkT, bool CS>
__device__ __forceinline__ void x2_site(float2* __restrict__ out, const float2* __restrict__ in,
                                        const LinkT* __restrict__ U, int nrhs, const StencilParams& P,
                                        const int* __restrict__ skip, int64_t site, int rhs0) {
    if (site >= P.vol || rhs0 >= nrhs) return;
    bool act[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) act[i] = rhs0 + i < nrhs && !(skip && skip[rhs0 + i]);
    if (!act[0] && !act[1]) return;
    const float2* fin = in + rhs0 * P.stride_rhs;
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
    float2 ar[12], ai[12];
    {
        Cx<float> pa[12], pb[12];
        if (act[0]) {
            Field<float>::load(fin, site, 2 * P.vol, pa);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) pa[k] = {0.f, 0.f};
        }
        if (act[1]) {
            Field<float>::load(fin + P.stride_rhs, site, 2 * P.vol, pb);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) pb[k] = {0.f, 0.f};
        }
        const float d = P.diag32;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            ar[k] = f2(d * pa[k].x, d * pb[k].x);
            ai[k] = f2(d * pa[k].y, d * pb[k].y);
        }
    }
    both_hops_x2<LinkT, 0>(ar, ai, fin, act, U, site, co, P);
    both_hops_x2<LinkT, 1>(ar, ai, fin, act, U, site, co, P);
    both_hops_x2<LinkT, 2>(ar, ai, fin, act, U, site, co, P);
    both_hops_x2<LinkT, 3>(ar, ai, fin, act, U, site, co, P);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (!act[i]) continue;
        Cx<float> o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float g5 = k < 6 ? 1.f : -1.f;  // gamma5 = diag(1, 1, -1, -1)
            o[k] = {g5 * (i ? ar[k].y : ar[k].x), g5 * (i ? ai[k].y : ai[k].x)};
        }
        Field<float>::template store<CS>(out + (rhs0 + i) * P.stride_rhs, site, 2 * P.vol, o);
    }
}

// Grid and thread layout as k_hw with NR = 2.
template <class LinkT, bool CS>
__device__ __forceinline__ void hw_x2_body(float2* __restrict__ out, const float2* __restrict__ in,
                                           const LinkT* __restrict__ U, int nrhs, const StencilParams& P,
                                           const int* __restrict__ skip, int ngrp) {
    const int64_t tile = blockIdx.x / (unsigned)ngrp;
    const int grp = (int)(blockIdx.x - tile * ngrp);
    x2_site<LinkT, CS>(out, in, U, nrhs, P, skip, tile * blockDim.x + threadIdx.x,
                       (grp * blockDim.y + threadIdx.y) * 2);
}

// The kernel as the compiler sizes it (144 registers: 12 warps per SM), and capped at 128
// registers (16 warps per SM, a few values spilled to local memory).
template <class LinkT, bool CS>
__global__ void __launch_bounds__(256)
    k_hw_x2(float2* __restrict__ out, const float2* __restrict__ in, const LinkT* __restrict__ U, int nrhs,
            StencilParams P, const int* __restrict__ skip, int ngrp) {
    hw_x2_body<LinkT, CS>(out, in, U, nrhs, P, skip, ngrp);
}
template <class LinkT, bool CS>
__global__ void __launch_bounds__(256, 2)
    k_hw_x2_r128(float2* __restrict__ out, const float2* __restrict__ in, const LinkT* __restrict__ U, int nrhs,
                 StencilParams P, const int* __restrict__ skip, int ngrp) {
    hw_x2_body<LinkT, CS>(out, in, U, nrhs, P, skip, ngrp);
}

// ---- pipelined FP32 form ------------------------------------------------------
// The same stencil with the neighbour spinors staged through shared memory:
// each thread copies its own next stage (the site itself, then the 8 hops)
// with cp.async while it computes the current one, so one stage of loads is
// always in flight per thread without holding registers for it.  Shared
// memory: 2 buffers x NR fields x 6 planes x 16 bytes per thread, thread-major
// (consecutive threads, consecutive 16-byte words: no bank conflicts).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int NR>
struct PipeCtx {
    float4* sbuf;
    int nthr, tid;
    const float2* in;
    int64_t stride_rhs, vol2;
    bool act[NR];
    __device__ __forceinline__ float4* slot(int buf, int i, int k) const {
        return sbuf + ((buf * NR + i) * 6 + k) * nthr + tid;
    }
    // stage `buf` <- the spinors of site nb of the NR fields
    __device__ __forceinline__ void issue(int buf, int nb) const {
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            if (!act[i]) continue;
            const float2* src = in + i * stride_rhs + 2 * (int64_t)nb;
#pragma unroll
            for (int k = 0; k < 6; ++k) cp_async16(slot(buf, i, k), src + k * vol2);
        }
    }
    __device__ __forceinline__ void read(int buf, int i, Cx<float> (&p)[12]) const {
        if (act[i]) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float4 v = *slot(buf, i, k);
                p[2 * k] = {v.x, v.y};
                p[2 * k + 1] = {v.z, v.w};
            }
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) p[k] = {0.f, 0.f};
        }
    }
};

// Site and coefficient of stage ST (0: the site itself; 2 nu + 1, 2 nu + 2: the forward
// and backward neighbour in direction nu), 32-bit site indices (vol < 2^27).
template <int ST>
__device__ __forceinline__ int stage_site(int site, const int (&co)[4], const StencilParams& P, float* coef) {
    if constexpr (ST == 0) {
        *coef = P.diag32;
        return site;
    } else {
        constexpr int NU = (ST - 1) / 2;
        int stride = 1;
#pragma unroll
        for (int d = 0; d < NU; ++d) stride *= P.L[d];
        const int L = P.L[NU];
        if constexpr (ST % 2) {  // forward
            float c = P.cf32[NU];
            int nb = site + stride;
            if (co[NU] == L - 1) {
                nb = site - (L - 1) * stride;
                if (P.ap[NU]) c = -c;
            }
            *coef = c;
            return nb;
        } else {  // backward
            float c = P.cb32[NU];
            int nb = site - stride;
            if (co[NU] == 0) {
                nb = site + (L - 1) * stride;
                if (P.ap[NU]) c = -c;
            }
            *coef = c;
            return nb;
        }
    }
}

// Stage ST (1..8) = hop NU = (ST - 1) / 2, forward (S = -1) for odd ST; its data sit in
// buffer ST % 2.  Before computing it, the next stage's copy is issued into the other
// buffer, which the previous stage finished reading.
template <class LinkT, int NR, int ST>
__device__ __forceinline__ void pipe_stage(Cx<float> (&acc)[NR][12], const PipeCtx<NR>& pc,
                                           const LinkT* __restrict__ U, int site, const int (&co)[4],
                                           const StencilParams& P) {
    constexpr int NU = (ST - 1) / 2;
    constexpr int S = (ST % 2) ? -1 : +1;
    if constexpr (ST < 8) {
        float unused;
        pc.issue((ST + 1) % 2, stage_site<ST + 1>(site, co, P, &unused));
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    float coef;
    const int nb = stage_site<ST>(site, co, P, &coef);
    Cx<float> h0[NR][3], h1[NR][3];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        Cx<float> p[12];
        pc.read(ST % 2, i, p);
        project<float, NU, S>(p, h0[i], h1[i]);
    }
    // forward hops use U_nu(site), backward ones U_nu(site - nu)^dag
    hop_links<float, LinkT, NU, S, NR>(acc, h0, h1, U, (ST % 2) ? site : nb, coef, P.vol);
}

template <class LinkT, int NR, bool CS>
__global__ void __launch_bounds__(256)
    k_hw_pipe(float2* __restrict__ out, const float2* __restrict__ in, const LinkT* __restrict__ U, int nrhs,
              StencilParams P, const int* __restrict__ skip, int ngrp) {
    extern __shared__ float4 sbuf[];
    const int64_t tile = blockIdx.x / (unsigned)ngrp;
    const int grp = (int)(blockIdx.x - tile * ngrp);
    const int64_t site = tile * blockDim.x + threadIdx.x;
    const int rhs0 = (grp * blockDim.y + threadIdx.y) * NR;
    if (site >= P.vol || rhs0 >= nrhs) return;  // no barrier below: early exit is safe
    PipeCtx<NR> pc;
    pc.sbuf = sbuf;
    pc.nthr = blockDim.x * blockDim.y;
    pc.tid = threadIdx.y * blockDim.x + threadIdx.x;
    pc.in = in + rhs0 * P.stride_rhs;
    pc.stride_rhs = P.stride_rhs;
    pc.vol2 = 2 * P.vol;
    bool any = false;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        pc.act[i] = rhs0 + i < nrhs && !(skip && skip[rhs0 + i]);
        any |= pc.act[i];
    }
    if (!any) return;
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
    const int s32 = (int)site;
    float c0;
    pc.issue(0, stage_site<0>(s32, co, P, &c0));
    cp_async_commit();
    {
        float unused;
        pc.issue(1, stage_site<1>(s32, co, P, &unused));
    }
    cp_async_commit();
    cp_async_wait<1>();
    Cx<float> acc[NR][12];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        pc.read(0, i, acc[i]);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[i][k] = scale(acc[i][k], c0);
    }
    pipe_stage<LinkT, NR, 1>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 2>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 3>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 4>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 5>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 6>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 7>(acc, pc, U, s32, co, P);
    pipe_stage<LinkT, NR, 8>(acc, pc, U, s32, co, P);
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        if (!pc.act[i]) continue;
#pragma unroll
        for (int k = 6; k < 12; ++k) acc[i][k] = {-acc[i][k].x, -acc[i][k].y};
        Field<float>::template store<CS>(out + (rhs0 + i) * P.stride_rhs, site, 2 * P.vol, acc[i]);
    }
}

// ---- colour-split FP32 form ---------------------------------------------------
// Three lanes per site and field, one per colour a = 0, 1, 2 (lanes 3 j + a of a warp
// for its 10 sites j; lanes 30 and 31 carry no site).  Lane a loads the four spin
// components of colour a of each neighbour (entries 3 s + a of the packed field),
// projects them to its colour of the half-spinor (1 -/+ gamma) psi, receives the other
// two colours from the lanes beside it (shuffles), multiplies them by row a of the
// link, U_ab h_b (forward) or conj(U_ba) h_b (backward), and accumulates the four spins
// of colour a.  A lane holds a quarter of the state of a one-field thread, so the
// kernel runs at about 50 registers and 40+ resident warps per SM, which keep far more
// loads in flight than the 12-16 warps of the two-field kernels.
// Grid: CTA b covers site tile b / ngrp and field group b % ngrp; warp w of the CTA
// takes site group tile * (warps / fw) + w / fw (10 sites) and field group * fw + w % fw.
constexpr int kCsSites = 10;  // sites per warp

__device__ __forceinline__ Cx<float> ldc(const float2* __restrict__ p) {
    const float2 v = __ldg(p);
    return {v.x, v.y};
}
__device__ __forceinline__ Cx<float> shfl_cx(Cx<float> v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
// acc += u * v (CONJ: conj(u) * v)
template <bool CONJ>
__device__ __forceinline__ void cmac_cs(Cx<float>& acc, Cx<float> u, Cx<float> v) {
    if constexpr (CONJ) cmac_conj(acc, u, v); else cmac(acc, u, v);
}

template <class LinkT, int NU, int S>
__device__ __forceinline__ void hop_cs(Cx<float> (&acc)[4], const float2* __restrict__ fin, int64_t vol2,
                                       bool act, const LinkT* __restrict__ U, int64_t link_site, int64_t nb,
                                       float coef, int64_t vol, int a, int a1, int a2, int src1, int src2) {
    // spins 0..3 of colour a at the neighbour: entry k = 3 s + a at (k/2) vol2 + 2 nb + k % 2
    Cx<float> p[4];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const int k = 3 * sp + a;
        p[sp] = act ? ldc(fin + (int64_t)(k >> 1) * vol2 + 2 * nb + (k & 1)) : Cx<float>{0.f, 0.f};
    }
    // this colour of the projected half-spinor h = psi_up + S B psi_dn
    const float sg = float(S);
    Cx<float> h0, h1;
    if constexpr (NU == 0) {  // B psi_dn = (-i p3, -i p2)
        h0 = p[0] + scale(mul_mi(p[3]), sg);
        h1 = p[1] + scale(mul_mi(p[2]), sg);
    } else if constexpr (NU == 1) {  // (-p3, p2)
        h0 = p[0] - scale(p[3], sg);
        h1 = p[1] + scale(p[2], sg);
    } else if constexpr (NU == 2) {  // (-i p2, i p3)
        h0 = p[0] + scale(mul_mi(p[2]), sg);
        h1 = p[1] + scale(mul_i(p[3]), sg);
    } else {  // (p2, p3)
        h0 = p[0] + scale(p[2], sg);
        h1 = p[1] + scale(p[3], sg);
    }
    // the two other colours from the lanes of the same site
    const Cx<float> h0b = shfl_cx(h0, src1), h1b = shfl_cx(h1, src1);
    const Cx<float> h0c = shfl_cx(h0, src2), h1c = shfl_cx(h1, src2);
    // row a of U(site) (forward) or of U(nb)^dag, i.e. column a of U(nb) conjugated (backward)
    const LinkT* lb = U + (int64_t)NU * 9 * vol + link_site;
    constexpr bool CJ = S > 0;
    auto uidx = [&](int b) -> int64_t { return (int64_t)(CJ ? 3 * b + a : 3 * a + b) * vol; };
    const Cx<float> ua = Link<float, LinkT>::ld(lb, uidx(a));
    const Cx<float> ub = Link<float, LinkT>::ld(lb, uidx(a1));
    const Cx<float> uc = Link<float, LinkT>::ld(lb, uidx(a2));
    Cx<float> g0 = {0.f, 0.f}, g1 = {0.f, 0.f};
    cmac_cs<CJ>(g0, ua, h0);
    cmac_cs<CJ>(g1, ua, h1);
    cmac_cs<CJ>(g0, ub, h0b);
    cmac_cs<CJ>(g1, ub, h1b);
    cmac_cs<CJ>(g0, uc, h0c);
    cmac_cs<CJ>(g1, uc, h1c);
    // reconstruction: upper spins coef g, lower spins coef S B^dag g
    const float cs = coef * sg;
    acc[0] = acc[0] + scale(g0, coef);
    acc[1] = acc[1] + scale(g1, coef);
    if constexpr (NU == 0) {  // B^dag g = (i g1, i g0)
        acc[2] = acc[2] + scale(mul_i(g1), cs);
        acc[3] = acc[3] + scale(mul_i(g0), cs);
    } else if constexpr (NU == 1) {  // (g1, -g0)
        acc[2] = acc[2] + scale(g1, cs);
        acc[3] = acc[3] - scale(g0, cs);
    } else if constexpr (NU == 2) {  // (i g0, -i g1)
        acc[2] = acc[2] + scale(mul_i(g0), cs);
        acc[3] = acc[3] + scale(mul_mi(g1), cs);
    } else {  // (g0, g1)
        acc[2] = acc[2] + scale(g0, cs);
        acc[3] = acc[3] + scale(g1, cs);
    }
}

template <class LinkT, int NU>
__device__ __forceinline__ void both_hops_cs(Cx<float> (&acc)[4], const float2* __restrict__ fin, bool act,
                                             const LinkT* __restrict__ U, int64_t site, const int co[4],
                                             const StencilParams& P, int a, int a1, int a2, int src1, int src2) {
    int64_t stride = 1;
#pragma unroll
    for (int d = 0; d < NU; ++d) stride *= P.L[d];
    const int L = P.L[NU];
    int64_t fw = site + stride;
    float cf = P.cf32[NU];
    if (co[NU] == L - 1) {
        fw = site - (int64_t)(L - 1) * stride;
        if (P.ap[NU]) cf = -cf;
    }
    int64_t bw = site - stride;
    float cb = P.cb32[NU];
    if (co[NU] == 0) {
        bw = site + (int64_t)(L - 1) * stride;
        if (P.ap[NU]) cb = -cb;
    }
    hop_cs<LinkT, NU, -1>(acc, fin, 2 * P.vol, act, U, site, fw, cf, P.vol, a, a1, a2, src1, src2);
    hop_cs<LinkT, NU, +1>(acc, fin, 2 * P.vol, act, U, bw, bw, cb, P.vol, a, a1, a2, src1, src2);
}

template <class LinkT, bool CS>
__global__ void __launch_bounds__(256, 4)
    k_hw_cs(float2* __restrict__ out, const float2* __restrict__ in, const LinkT* __restrict__ U, int nrhs,
            StencilParams P, const int* __restrict__ skip, int ngrp, int fw) {
    const int warp = threadIdx.y, lane = threadIdx.x;
    const int64_t tile = blockIdx.x / (unsigned)ngrp;
    const int grp = (int)(blockIdx.x - tile * ngrp);
    const int sgpc = blockDim.y / fw;  // site groups per CTA
    const int64_t sgroup = tile * sgpc + warp / fw;
    const int field = grp * fw + warp % fw;
    // warp-uniform exits only (every lane of a warp takes part in the shuffles)
    if (field >= nrhs || (skip && skip[field])) return;
    if (sgroup * kCsSites >= P.vol) return;
    const int j = lane / 3;
    const int a = lane - 3 * j;           // colour of this lane (lanes 30, 31: j = 10, a = 0, 1)
    const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
    const int jj = j < kCsSites ? j : kCsSites - 1;
    const int src1 = 3 * jj + a1, src2 = 3 * jj + a2;
    const int64_t site0 = sgroup * kCsSites + jj;
    const bool act = j < kCsSites && site0 < P.vol;
    const int64_t site = act ? site0 : sgroup * kCsSites;  // idle lanes: a valid site, nothing stored
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
    const float2* fin = in + (int64_t)field * P.stride_rhs;
    const int64_t vol2 = 2 * P.vol;
    Cx<float> acc[4];
    const float d = P.diag32;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const int k = 3 * sp + a;
        acc[sp] = act ? scale(ldc(fin + (int64_t)(k >> 1) * vol2 + 2 * site + (k & 1)), d) : Cx<float>{0.f, 0.f};
    }
    both_hops_cs<LinkT, 0>(acc, fin, act, U, site, co, P, a, a1, a2, src1, src2);
    both_hops_cs<LinkT, 1>(acc, fin, act, U, site, co, P, a, a1, a2, src1, src2);
    both_hops_cs<LinkT, 2>(acc, fin, act, U, site, co, P, a, a1, a2, src1, src2);
    both_hops_cs<LinkT, 3>(acc, fin, act, U, site, co, P, a, a1, a2, src1, src2);
    if (!act) return;
    float2* fo = out + (int64_t)field * P.stride_rhs;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const int k = 3 * sp + a;
        const float g5 = sp < 2 ? 1.f : -1.f;  // gamma5 = diag(1, 1, -1, -1)
        const float2 v = make_float2(g5 * acc[sp].x, g5 * acc[sp].y);
        float2* dst = fo + (int64_t)(k >> 1) * vol2 + 2 * site + (k & 1);
        if constexpr (CS) __stcs(dst, v); else *dst = v;
    }
}

// ---- layout conversions (one thread per site of one field) --------------------
template <class T>
__global__ void k_pack(const T* __restrict__ in, T* __restrict__ out, int64_t vol) {
    const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= vol) return;
    const int64_t f = (int64_t)blockIdx.y * 12 * vol;
    const T* src = in + f + site * 12;
    T* dst = out + f + 2 * site;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        dst[k * 2 * vol] = src[2 * k];
        dst[k * 2 * vol + 1] = src[2 * k + 1];
    }
}
template <class T>
__global__ void k_unpack(const T* __restrict__ in, T* __restrict__ out, int64_t vol) {
    const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= vol) return;
    const int64_t f = (int64_t)blockIdx.y * 12 * vol;
    const T* src = in + f + 2 * site;
    T* dst = out + f + site * 12;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        dst[2 * k] = src[k * 2 * vol];
        dst[2 * k + 1] = src[k * 2 * vol + 1];
    }
}
__global__ void k_pack_links(const double2* __restrict__ in, double2* __restrict__ out, int64_t vol) {
    const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= vol) return;
#pragma unroll 4
    for (int e = 0; e < 36; ++e) out[e * vol + site] = in[site * 36 + e];
}

template <class R, class LinkT, int NR>
cudaError_t launch_nr(typename Field<R>::T* out, const typename Field<R>::T* in, const LinkT* U, int nrhs,
                      const StencilParams& p, const int* skip, cudaStream_t st, int sx, int rb) {
    const int groups = (nrhs + NR - 1) / NR;
    const int ngrp = (groups + rb - 1) / rb;
    const int64_t tiles = (p.vol + sx - 1) / sx;
    if (tiles * ngrp > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 block(sx, rb);
    const bool cs = (double)nrhs * (double)p.vol * 12.0 * sizeof(typename Field<R>::T) > 256.0 * (1 << 20);
    if (cs)
        k_hw<R, LinkT, NR, true><<<(unsigned)(tiles * ngrp), block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp);
    else
        k_hw<R, LinkT, NR, false><<<(unsigned)(tiles * ngrp), block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp);
    count_launch();
    return cudaGetLastError();
}

template <class LinkT, int NR>
cudaError_t launch_pipe(float2* out, const float2* in, const LinkT* U, int nrhs, const StencilParams& p,
                        const int* skip, cudaStream_t st, int sx, int rb) {
    const int groups = (nrhs + NR - 1) / NR;
    const int ngrp = (groups + rb - 1) / rb;
    const int64_t tiles = (p.vol + sx - 1) / sx;
    if (tiles * ngrp > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * NR * 6 * sizeof(float4) * sx * rb;
    const bool cs = (double)nrhs * (double)p.vol * 12.0 * sizeof(float2) > 256.0 * (1 << 20);
    // opt in to more than 48 KB of dynamic shared memory, once per kernel and device
    static bool opted[2][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const int maxs = 2 * 2 * 6 * (int)sizeof(float4) * 256;
    if (!opted[cs][dev]) {
        e = cs ? cudaFuncSetAttribute(k_hw_pipe<LinkT, NR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs)
               : cudaFuncSetAttribute(k_hw_pipe<LinkT, NR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
        if (e != cudaSuccess) return e;
        opted[cs][dev] = true;
    }
    dim3 block(sx, rb);
    if (cs)
        k_hw_pipe<LinkT, NR, true><<<(unsigned)(tiles * ngrp), block, smem, st>>>(out, in, U, nrhs, p, skip, ngrp);
    else
        k_hw_pipe<LinkT, NR, false><<<(unsigned)(tiles * ngrp), block, smem, st>>>(out, in, U, nrhs, p, skip, ngrp);
    count_launch();
    return cudaGetLastError();
}

// Colour-split kernel: CTA = 32 lanes x (sg site groups x fw fields) warps.
template <class LinkT>
cudaError_t launch_cs(float2* out, const float2* in, const LinkT* U, int nrhs, const StencilParams& p, const int* skip,
                      cudaStream_t st, int sg, int fw) {
    if (sg < 1 || fw < 1 || sg * fw > 8) return cudaErrorInvalidValue;
    const int ngrp = (nrhs + fw - 1) / fw;
    const int64_t groups = (p.vol + kCsSites - 1) / kCsSites;
    const int64_t tiles = (groups + sg - 1) / sg;
    if (tiles * ngrp > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 block(32, sg * fw);
    const bool cs = (double)nrhs * (double)p.vol * 12.0 * sizeof(float2) > 256.0 * (1 << 20);
    const unsigned grid = (unsigned)(tiles * ngrp);
    if (cs)
        k_hw_cs<LinkT, true><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp, fw);
    else
        k_hw_cs<LinkT, false><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp, fw);
    count_launch();
    return cudaGetLastError();
}

template <class LinkT, int MINB>
cudaError_t launch_x2(float2* out, const float2* in, const LinkT* U, int nrhs, const StencilParams& p,
                      const int* skip, cudaStream_t st, int sx, int rb) {
    const int groups = (nrhs + 1) / 2;
    const int ngrp = (groups + rb - 1) / rb;
    const int64_t tiles = (p.vol + sx - 1) / sx;
    if (tiles * ngrp > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 block(sx, rb);
    const bool cs = (double)nrhs * (double)p.vol * 12.0 * sizeof(float2) > 256.0 * (1 << 20);
    const unsigned grid = (unsigned)(tiles * ngrp);
    if (MINB == 2) {
        if (cs)
            k_hw_x2_r128<LinkT, true><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp);
        else
            k_hw_x2_r128<LinkT, false><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp);
    } else if (cs) {
        k_hw_x2<LinkT, true><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp);
    } else {
        k_hw_x2<LinkT, false><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip, ngrp);
    }
    count_launch();
    return cudaGetLastError();
}

template <class R, class LinkT>
cudaError_t launch(typename Field<R>::T* out, const typename Field<R>::T* in, const LinkT* U, int nrhs,
                   const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh) {
    if (nrhs <= 0 || p.vol <= 0) return cudaSuccess;
    if (sh.pipe == 4) {  // the colour-split FP32 kernel: sx site groups of 10 sites, rb fields per CTA
        if constexpr (sizeof(R) == 4) {
            if (sh.nr != 1) return cudaErrorInvalidValue;
            return launch_cs<LinkT>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (sh.pipe == 2 || sh.pipe == 3) {  // the paired FP32 kernel (3: capped at 128 registers)
        if constexpr (sizeof(R) == 4) {
            if (sh.sx % 32 != 0 || sh.rb < 1 || sh.sx * sh.rb > 256 || sh.nr != 2) return cudaErrorInvalidValue;
            if (sh.pipe == 3) return launch_x2<LinkT, 2>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
            return launch_x2<LinkT, 1>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (sh.pipe) {  // the pipelined FP32 kernel: 1 or 2 fields per thread, up to 256 threads per CTA
        if constexpr (sizeof(R) == 4) {
            if (sh.sx % 32 != 0 || sh.rb < 1 || sh.sx * sh.rb > 256 || sh.nr < 1 || sh.nr > 2)
                return cudaErrorInvalidValue;
            if (sh.nr == 1) return launch_pipe<LinkT, 1>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
            return launch_pipe<LinkT, 2>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (sh.sx > 0 && sh.rb > 0) {  // a tuned shape: validate it against the kernel's launch bounds
        const int maxnr = sizeof(R) == 8 ? 1 : 3;  // more fields per thread spill registers
        if (sh.sx % 32 != 0 || sh.nr < 1 || sh.nr > maxnr || sh.sx * sh.rb > (sh.nr == 1 ? 384 : 256))
            return cudaErrorInvalidValue;
        if constexpr (sizeof(R) == 4) {
            if (sh.nr == 2) return launch_nr<R, LinkT, 2>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
            if (sh.nr == 3) return launch_nr<R, LinkT, 3>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
        }
        return launch_nr<R, LinkT, 1>(out, in, U, nrhs, p, skip, st, sh.sx, sh.rb);
    }
    // default: one field per thread, up to 12 fields of a site tile per CTA
    int rb = nrhs <= 12 ? nrhs : 8;
    int sx = 256 / rb;
    sx = sx < 32 ? 32 : (sx / 32) * 32;
    if (sx * rb > 384) sx = 32;
    return launch_nr<R, LinkT, 1>(out, in, U, nrhs, p, skip, st, sx, rb);
}

}  // namespace

template <class T>
cudaError_t pack_fields(const T* natural, T* packed, int64_t vol, int nfield, cudaStream_t st) {
    if (nfield <= 0 || vol <= 0) return cudaSuccess;
    if (nfield > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((vol + 255) / 256), (unsigned)nfield);
    k_pack<T><<<grid, 256, 0, st>>>(natural, packed, vol);
    count_launch();
    return cudaGetLastError();
}
template <class T>
cudaError_t unpack_fields(const T* packed, T* natural, int64_t vol, int nfield, cudaStream_t st) {
    if (nfield <= 0 || vol <= 0) return cudaSuccess;
    if (nfield > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((vol + 255) / 256), (unsigned)nfield);
    k_unpack<T><<<grid, 256, 0, st>>>(packed, natural, vol);
    count_launch();
    return cudaGetLastError();
}
template cudaError_t pack_fields<double2>(const double2*, double2*, int64_t, int, cudaStream_t);
template cudaError_t pack_fields<float2>(const float2*, float2*, int64_t, int, cudaStream_t);
template cudaError_t unpack_fields<double2>(const double2*, double2*, int64_t, int, cudaStream_t);
template cudaError_t unpack_fields<float2>(const float2*, float2*, int64_t, int, cudaStream_t);

cudaError_t pack_links(const double2* natural, double2* packed, int64_t vol, cudaStream_t st) {
    k_pack_links<<<(unsigned)((vol + 255) / 256), 256, 0, st>>>(natural, packed, vol);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hw_f64(double2* out, const double2* in, const double2* U, int nrhs, const StencilParams& p,
                          const int* skip, cudaStream_t st, StencilShape sh) {
    return launch<double, double2>(out, in, U, nrhs, p, skip, st, sh);
}
cudaError_t launch_hw_f32(float2* out, const float2* in, const float2* U, int nrhs, const StencilParams& p,
                          const int* skip, cudaStream_t st, StencilShape sh) {
    return launch<float, float2>(out, in, U, nrhs, p, skip, st, sh);
}
cudaError_t launch_hw_f32_bf16links(float2* out, const float2* in, const __nv_bfloat162* U, int nrhs,
                                    const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh) {
    return launch<float, __nv_bfloat162>(out, in, U, nrhs, p, skip, st, sh);
}
cudaError_t launch_hw_f32_f16links(float2* out, const float2* in, const __half2* U, int nrhs,
                                   const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh) {
    return launch<float, __half2>(out, in, U, nrhs, p, skip, st, sh);
}

}  // namespace sgn
