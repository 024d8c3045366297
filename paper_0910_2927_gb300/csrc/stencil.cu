// Wilson kernel H_W(mu) = gamma5 D_W(mu) on nrhs fields (Sec. 1 of the paper;
// D_W(mu) with e^{+mu} on forward and e^{-mu} on backward time hops).
//
// One thread computes one site of one field.  A CTA covers SX consecutive
// sites (x fastest) for RB fields, so the RB warps that share a site tile
// read the same links back to back and the link bytes come from L1 after the
// first field: with 12 fields the links cost 1/12 of their bytes per field.
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
template <class R>
struct Field;
template <>
struct Field<double> {
    using T = double2;
    static __device__ __forceinline__ void load(const double2* __restrict__ f, int64_t site, Cx<double> p[12]) {
        const double2* s = f + site * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = __ldg(s + k);
            p[k] = {v.x, v.y};
        }
    }
    static __device__ __forceinline__ void store(double2* __restrict__ f, int64_t site, const Cx<double> p[12]) {
        double2* s = f + site * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = make_double2(p[k].x, p[k].y);
    }
};
template <>
struct Field<float> {
    using T = float2;
    static __device__ __forceinline__ void load(const float2* __restrict__ f, int64_t site, Cx<float> p[12]) {
        const float4* s = reinterpret_cast<const float4*>(f + site * 12);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = __ldg(s + k);
            p[2 * k] = {v.x, v.y};
            p[2 * k + 1] = {v.z, v.w};
        }
    }
    static __device__ __forceinline__ void store(float2* __restrict__ f, int64_t site, const Cx<float> p[12]) {
        float4* s = reinterpret_cast<float4*>(f + site * 12);
#pragma unroll
        for (int k = 0; k < 6; ++k) s[k] = make_float4(p[2 * k].x, p[2 * k].y, p[2 * k + 1].x, p[2 * k + 1].y);
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

// One hop: acc += coef * (1 + S gamma_NU) W psi(nb), W = U_NU(site) (forward,
// S = -1) or U_NU(nb)^dag (backward, S = +1).  Spin index a*3 + colour c.
//   (1 + S gamma) psi = [h ; S B^dag h],  h = psi_up + S B psi_dn,
//   gamma_NU = [[0, B], [B^dag, 0]]:  B = -i sigma_{x,y,z}, or 1 for t.
template <class R, class LinkT, int NU, int S>
__device__ __forceinline__ void hop(Cx<R> acc[12], const typename Field<R>::T* __restrict__ in,
                                    const LinkT* __restrict__ U, int64_t link_site, int64_t nb, R coef) {
    Cx<R> p[12];
    Field<R>::load(in, nb, p);
    Cx<R> h0[3], h1[3];
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
    const int64_t lb = (link_site * 4 + NU) * 9;
    Cx<R> g0[3], g1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g0[a] = {R(0), R(0)};
        g1[a] = {R(0), R(0)};
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if constexpr (S < 0) {  // U(site) h
                Cx<R> u = Link<R, LinkT>::ld(U, lb + a * 3 + b);
                cmac(g0[a], u, h0[b]);
                cmac(g1[a], u, h1[b]);
            } else {  // U(nb)^dag h: (U^dag)_{ab} = conj(U_{ba})
                Cx<R> u = Link<R, LinkT>::ld(U, lb + b * 3 + a);
                cmac_conj(g0[a], u, h0[b]);
                cmac_conj(g1[a], u, h1[b]);
            }
        }
    }
    const R cs = coef * s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = acc[c] + scale(g0[c], coef);
        acc[3 + c] = acc[3 + c] + scale(g1[c], coef);
        if constexpr (NU == 0) {  // B^dag g = (i g1, i g0)
            acc[6 + c] = acc[6 + c] + scale(mul_i(g1[c]), cs);
            acc[9 + c] = acc[9 + c] + scale(mul_i(g0[c]), cs);
        } else if constexpr (NU == 1) {  // (g1, -g0)
            acc[6 + c] = acc[6 + c] + scale(g1[c], cs);
            acc[9 + c] = acc[9 + c] - scale(g0[c], cs);
        } else if constexpr (NU == 2) {  // (i g0, -i g1)
            acc[6 + c] = acc[6 + c] + scale(mul_i(g0[c]), cs);
            acc[9 + c] = acc[9 + c] + scale(mul_mi(g1[c]), cs);
        } else {  // (g0, g1)
            acc[6 + c] = acc[6 + c] + scale(g0[c], cs);
            acc[9 + c] = acc[9 + c] + scale(g1[c], cs);
        }
    }
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

template <class R, class LinkT, int NU>
__device__ __forceinline__ void both_hops(Cx<R> acc[12], const typename Field<R>::T* __restrict__ in,
                                          const LinkT* __restrict__ U, int64_t site, const int co[4],
                                          const StencilParams& P) {
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
    hop<R, LinkT, NU, -1>(acc, in, U, site, fw, cf);
    hop<R, LinkT, NU, +1>(acc, in, U, bw, bw, cb);
}

template <class R, class LinkT>
__global__ void __launch_bounds__(384) k_hw(typename Field<R>::T* __restrict__ out,
                                            const typename Field<R>::T* __restrict__ in,
                                            const LinkT* __restrict__ U, int nrhs, StencilParams P,
                                            const int* __restrict__ skip) {
    const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y * blockDim.y + threadIdx.y;
    if (site >= P.vol || rhs >= nrhs) return;
    if (skip && skip[rhs]) return;
    const typename Field<R>::T* fin = in + rhs * P.stride_rhs;
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
    Cx<R> acc[12];
    {
        Field<R>::load(fin, site, acc);
        const R d = diag_of<R>(P);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = scale(acc[k], d);
    }
    both_hops<R, LinkT, 0>(acc, fin, U, site, co, P);
    both_hops<R, LinkT, 1>(acc, fin, U, site, co, P);
    both_hops<R, LinkT, 2>(acc, fin, U, site, co, P);
    both_hops<R, LinkT, 3>(acc, fin, U, site, co, P);
    // gamma5 = diag(1, 1, -1, -1)
#pragma unroll
    for (int k = 6; k < 12; ++k) acc[k] = {-acc[k].x, -acc[k].y};
    Field<R>::store(out + rhs * P.stride_rhs, site, acc);
}

template <class R, class LinkT>
cudaError_t launch(typename Field<R>::T* out, const typename Field<R>::T* in, const LinkT* U, int nrhs,
                   const StencilParams& p, const int* skip, cudaStream_t st, StencilShape sh) {
    if (nrhs <= 0 || p.vol <= 0) return cudaSuccess;
    int rb = nrhs <= 12 ? nrhs : 8;
    int sx = 256 / rb;
    sx = sx < 32 ? 32 : (sx / 32) * 32;
    if (sx * rb > 384) sx = 32;
    if (sh.sx > 0 && sh.rb > 0 && sh.sx % 32 == 0 && sh.sx * sh.rb <= 384) {
        sx = sh.sx;
        rb = sh.rb;
    }
    dim3 block(sx, rb);
    dim3 grid((unsigned)((p.vol + sx - 1) / sx), (unsigned)((nrhs + rb - 1) / rb));
    k_hw<R, LinkT><<<grid, block, 0, st>>>(out, in, U, nrhs, p, skip);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

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

}  // namespace sgn
