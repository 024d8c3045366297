// The small dense steps of Algorithm 1, kept on the device:
//   y_i = beta rho_i (H_k - sigma_i I)^{-1} e_1          (one warp per column and shift)
//   rho_i <- -h_{k+1,k} e_k^T y_i                        (collinearity factor, eq. (3.1))
//   c = sum_i omega_i y_i                                (the combination of eq. (2.3))
// The shifted Hessenberg systems are solved by Gaussian elimination with
// partial pivoting: on a Hessenberg matrix the pivot of column r is chosen
// between the running row r and the untouched row r+1 (larger modulus, the
// running row on ties), and each lane of the warp owns two matrix columns.
#include "blas.cuh"

namespace sgn {
namespace {

constexpr int KMAX = 64;

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 shfl(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// BORDER = false: FOM, (H_k - sigma_i I) y = beta rho_i e_1 (k x k), shift i = blockIdx.x.
// BORDER = true: the non-seed shifts of restarted multishift GMRES, shift i = blockIdx.x + 1:
// [Hbar_k - sigma_i I~ | z] (y, tau) = beta rho_i e_1, (k+1) x (k+1), z = gres the seed's
// residual coefficients; the new residual of shift i is tau times the seed's, so rho_i <- tau.
// Both matrices are upper Hessenberg (the bordered one has a full last column), so the
// same adjacent-row pivoting applies.
template <bool BORDER>
__global__ void __launch_bounds__(32) k_shifted_solve(DevState S) {
    const int i = BORDER ? blockIdx.x + 1 : blockIdx.x;  // shift
    const int col = blockIdx.y;  // column
    if (S.done[col]) return;
    const int lane = threadIdx.x;
    const int km = S.kmax;
    const int kk = S.kk[col];
    const int q = BORDER ? kk + 1 : kk;    // system size
    const int ld = BORDER ? km + 1 : km;   // row stride of U
    const double2* H = S.H + (int64_t)col * (km + 1) * km;
    const double2* z = BORDER ? S.gres + (int64_t)col * (km + 1) : nullptr;
    const double sigma = S.sigma[(int64_t)col * S.s + i];
    const double sigma_im = S.sigma_im ? S.sigma_im[(int64_t)col * S.s + i] : 0.0;
    extern __shared__ double2 U[];  // [q][ld] upper factor, row-major
    __shared__ double2 zU[KMAX + 1];
    const int c0 = lane, c1 = lane + 32, c2 = lane + 64;  // c2: only the bordered column 64
    auto Hm = [&](int r, int c) -> double2 {  // system matrix entry (r, c)
        if (BORDER && c == kk) return z[r];
        double2 h = H[(int64_t)r * km + c];
        if (r == c) {
            h.x -= sigma;
            h.y -= sigma_im;
        }
        return h;
    };
    double2 w0 = c0 < q ? Hm(0, c0) : make_double2(0, 0);
    double2 w1 = c1 < q ? Hm(0, c1) : make_double2(0, 0);
    double2 w2 = c2 < q ? Hm(0, c2) : make_double2(0, 0);
    const double beta = S.beta[col];
    const double2 rho = S.rho[(int64_t)col * S.s + i];
    double2 zw = make_double2(beta * rho.x, beta * rho.y);
    bool singular = false;
    for (int r = 0; r < q; ++r) {
        const int owner = r & 31;
        double2 a = shfl(r >= 64 ? w2 : (r >= 32 ? w1 : w0), owner);
        if (r == q - 1) {
            if (c0 >= r && c0 < q) U[r * ld + c0] = w0;
            if (c1 >= r && c1 < q) U[r * ld + c1] = w1;
            if (c2 >= r && c2 < q) U[r * ld + c2] = w2;
            if (lane == 0) zU[r] = zw;
            if (a.x == 0 && a.y == 0) singular = true;
            break;
        }
        double2 n0 = (c0 >= r && c0 < q) ? Hm(r + 1, c0) : make_double2(0, 0);
        double2 n1 = (c1 >= r && c1 < q) ? Hm(r + 1, c1) : make_double2(0, 0);
        double2 n2 = (c2 >= r && c2 < q) ? Hm(r + 1, c2) : make_double2(0, 0);
        double2 b = Hm(r + 1, r);
        const bool swap = cabs2(b) > cabs2(a);  // row r+1 becomes the pivot row
        double2 p0 = swap ? n0 : w0, p1 = swap ? n1 : w1, p2 = swap ? n2 : w2;
        double2 o0 = swap ? w0 : n0, o1 = swap ? w1 : n1, o2 = swap ? w2 : n2;
        double2 zp = swap ? make_double2(0, 0) : zw, zo = swap ? zw : make_double2(0, 0);
        double2 piv = swap ? b : a;
        double2 oth = swap ? a : b;
        if (piv.x == 0 && piv.y == 0) {
            singular = true;
            break;
        }
        double2 l = cdiv(oth, piv);
        if (c0 >= r && c0 < q) U[r * ld + c0] = p0;
        if (c1 >= r && c1 < q) U[r * ld + c1] = p1;
        if (c2 >= r && c2 < q) U[r * ld + c2] = p2;
        if (lane == 0) zU[r] = zp;
        w0 = c0 > r ? csub(o0, cmul(l, p0)) : make_double2(0, 0);
        w1 = c1 > r ? csub(o1, cmul(l, p1)) : make_double2(0, 0);
        w2 = c2 > r ? csub(o2, cmul(l, p2)) : make_double2(0, 0);
        zw = csub(zo, cmul(l, zp));
    }
    double2* y = S.y + ((int64_t)col * S.s + i) * km;
    if (singular) {
        if (lane == 0) atomicOr(S.err, 1);
        for (int j = lane; j < km; j += 32) y[j] = make_double2(0, 0);
        return;
    }
    __syncwarp();
    // column-oriented back substitution; lane owns rows lane, lane + 32 (and lane + 64)
    double2 z0 = c0 < q ? zU[c0] : make_double2(0, 0);
    double2 z1 = c1 < q ? zU[c1] : make_double2(0, 0);
    double2 z2 = c2 < q ? zU[c2] : make_double2(0, 0);
    double2 ylast = make_double2(0, 0);
    for (int r = q - 1; r >= 0; --r) {
        const int owner = r & 31;
        double2 zr = shfl(r >= 64 ? z2 : (r >= 32 ? z1 : z0), owner);
        double2 yr = cdiv(zr, U[r * ld + r]);
        if (r == q - 1) ylast = yr;
        if (lane == owner && r < kk) y[r] = yr;
        if (c0 < r) z0 = csub(z0, cmul(U[c0 * ld + r], yr));
        if (c1 < r) z1 = csub(z1, cmul(U[c1 * ld + r], yr));
        if (c2 < r) z2 = csub(z2, cmul(U[c2 * ld + r], yr));
    }
    for (int j = kk + lane; j < km; j += 32) y[j] = make_double2(0, 0);
    if (lane == 0) {
        double2 rnew = make_double2(0, 0);
        if (BORDER) {
            rnew = ylast;  // tau
        } else if (kk == km) {
            double2 h = H[(int64_t)kk * km + (kk - 1)];
            rnew = cmul(h, ylast);
            rnew.x = -rnew.x;
            rnew.y = -rnew.y;
        }
        S.rho[(int64_t)col * S.s + i] = rnew;
    }
}

__global__ void k_combine(DevState S) {
    const int col = blockIdx.x;
    if (S.done[col]) return;
    const int km = S.kmax;
    for (int j = threadIdx.x; j < km; j += blockDim.x) {
        double2 c = make_double2(0, 0);
        for (int i = 0; i < S.s; ++i) {
            double2 y = S.y[((int64_t)col * S.s + i) * km + j];
            double w = S.omega[(int64_t)col * S.s + i];
            c.x = fma(w, y.x, c.x);
            c.y = fma(w, y.y, c.y);
        }
        S.coef[(int64_t)col * S.rstride + j] = c;
    }
}

// Minimal-residual form for one shift per column (restarted GMRES):  y = argmin
// || beta rho e_1 - (Hbar_k - sigma I~) y ||  by Givens rotations, with the
// coefficients of the new residual, c = beta rho e_1 - (Hbar_k - sigma I~) y, in
// gres[col][0..kk] (the next restart vector is V_{k+1} c) and rho = 1.  One CTA per
// column; the rotations run on one thread over a shared-memory copy (k <= 64:
// O(k^2) work, once per cycle).
__global__ void k_shifted_lsq(DevState S) {
    const int col = blockIdx.x;
    if (S.done[col] || threadIdx.x != 0) return;
    const int km = S.kmax;
    const int kk = S.kk[col];
    const double2* H = S.H + (int64_t)col * (km + 1) * km;
    const double sig = S.sigma[(int64_t)col * S.s];
    const double sig_im = S.sigma_im ? S.sigma_im[(int64_t)col * S.s] : 0.0;
    extern __shared__ double2 M[];  // [(kk + 1)][km]
    __shared__ double2 g[KMAX + 1];
    for (int r = 0; r <= kk; ++r)
        for (int c = 0; c < kk; ++c) {
            double2 h = H[(int64_t)r * km + c];
            if (r == c) {
                h.x -= sig;
                h.y -= sig_im;
            }
            M[r * km + c] = h;
        }
    const double beta = S.beta[col];
    const double2 rho = S.rho[(int64_t)col * S.s];
    const double2 b0 = make_double2(beta * rho.x, beta * rho.y);
    for (int r = 0; r <= kk; ++r) g[r] = r == 0 ? b0 : make_double2(0, 0);
    // rows c and c+1: G = [[conj(cs), conj(sn)], [-sn, cs]] zeroes M[c+1][c]
    for (int c = 0; c < kk; ++c) {
        const double2 a = M[c * km + c], b = M[(c + 1) * km + c];
        const double nr = sqrt(cabs2(a) + cabs2(b));
        if (!(nr > 0)) continue;  // zero column (only at a breakdown): y_c = 0 below
        const double2 cs = make_double2(a.x / nr, a.y / nr), sn = make_double2(b.x / nr, b.y / nr);
        for (int j = c; j < kk; ++j) {
            const double2 x = M[c * km + j], y = M[(c + 1) * km + j];
            M[c * km + j] = cadd(cconjmul(cs, x), cconjmul(sn, y));
            M[(c + 1) * km + j] = csub(cmul(cs, y), cmul(sn, x));
        }
        const double2 x = g[c], y = g[c + 1];
        g[c] = cadd(cconjmul(cs, x), cconjmul(sn, y));
        g[c + 1] = csub(cmul(cs, y), cmul(sn, x));
    }
    double2* yv = S.y + (int64_t)col * S.s * km;
    for (int r = kk - 1; r >= 0; --r) {
        double2 z = g[r];
        for (int j = r + 1; j < kk; ++j) z = csub(z, cmul(M[r * km + j], yv[j]));
        const double2 d = M[r * km + r];
        const double dd = cabs2(d);
        yv[r] = dd > 0 ? make_double2((z.x * d.x + z.y * d.y) / dd, (z.y * d.x - z.x * d.y) / dd) : make_double2(0, 0);
    }
    for (int j = kk; j < km; ++j) yv[j] = make_double2(0, 0);
    // c = beta rho e_1 - (Hbar - sigma I~) y, from the unrotated matrix
    double2* cres = S.gres + (int64_t)col * (km + 1);
    for (int r = 0; r <= km; ++r) {
        double2 acc = r == 0 ? b0 : make_double2(0, 0);
        if (r <= kk)
            for (int c = (r > 0 ? r - 1 : 0); c < kk; ++c) {
                double2 h = H[(int64_t)r * km + c];
                if (r == c) {
                    h.x -= sig;
                    h.y -= sig_im;
                }
                acc = csub(acc, cmul(h, yv[c]));
            }
        cres[r] = acc;
    }
    S.rho[(int64_t)col * S.s] = make_double2(1, 0);
}

}  // namespace

cudaError_t shifted_lsq(const DevState& S, int ncol, cudaStream_t st) {
    if (S.s < 1 || !S.gres || S.kmax > KMAX) return cudaErrorInvalidValue;
    k_shifted_lsq<<<ncol, 32, sizeof(double2) * (S.kmax + 1) * S.kmax, st>>>(S);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || S.s == 1) return e;
    // the other shifts: bordered systems with the seed's residual coefficients
    k_shifted_solve<true><<<dim3(S.s - 1, ncol), 32, sizeof(double2) * (S.kmax + 1) * (S.kmax + 1), st>>>(S);
    count_launch();
    return cudaGetLastError();
}

cudaError_t prepare_small_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_shifted_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double2) * KMAX * KMAX));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_shifted_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(double2) * (KMAX + 1) * (KMAX + 1)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_shifted_lsq, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double2) * (KMAX + 1) * KMAX));
}

cudaError_t shifted_solves(const DevState& S, int ncol, cudaStream_t st) {
    if (S.kmax > KMAX) return cudaErrorInvalidValue;
    size_t smem = sizeof(double2) * (size_t)S.kmax * S.kmax;
    k_shifted_solve<false><<<dim3(S.s, ncol), 32, smem, st>>>(S);
    count_launch();
    return cudaGetLastError();
}

cudaError_t combine_shifts(const DevState& S, int ncol, cudaStream_t st) {
    k_combine<<<ncol, 64, 0, st>>>(S);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sgn
