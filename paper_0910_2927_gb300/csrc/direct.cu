// The direct projection that the paper compares Algorithm 1 against (Sec. 6, eq. (6.3)):
//   x = x_P + ||r|| V_k sign(H_k) e_1,   r = (I - P) b,   x_P = R sign(Re Lambda) L^dag b,
// with V_k, H_k from k Arnoldi steps on A itself (no rational approximation, no restarts),
// and sign(H_k) by Roberts' Newton iteration X <- (X + X^{-1}) / 2 on the k x k matrix.
// The whole basis is kept (k + 1 FP64 fields per column, the method's memory cost); the
// Arnoldi steps use the FP64 stencil and two classical Gram-Schmidt passes, in blocks of at
// most 128 basis vectors per kernel (the reduction's slot limit).  The Newton iterations run
// on the GPU for all columns at once: X^{-1} by Gauss-Jordan elimination with partial
// pivoting on [X | I], one launch pair per pivot (captured once as a CUDA graph), with the
// matrices of shorter Krylov dimension padded by the identity (sign(I) = I).
#include "ctx.cuh"
#include "dense_eig.h"

#include <algorithm>

namespace sgn {

namespace {
constexpr int GS_BLOCK = 128;
using cdd = std::complex<double>;

__device__ __forceinline__ double2 cdiv_d(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// Gauss-Jordan step p on the augmented matrices A[col] = [X | I] (q rows, 2q columns,
// row-major): pivot row = the first row i >= p of largest |A[i][p]|, swapped with row p,
// row p scaled by 1 / pivot, and the column of elimination factors A[i][p] saved to fac.
// One CTA per matrix.  A zero pivot (singular X: an eigenvalue of H_k on the imaginary
// axis) sets bad[col].
__global__ void __launch_bounds__(256) k_gj_pivot(double2* __restrict__ A, int q, int p, double2* __restrict__ fac,
                                                  int* __restrict__ bad) {
    const int col = blockIdx.x;
    double2* M = A + (size_t)col * q * 2 * q;
    const int ld = 2 * q;
    __shared__ double sv[256];
    __shared__ int si[256];
    double best = -1.0;
    int bi = p;
    for (int i = p + threadIdx.x; i < q; i += blockDim.x) {
        const double2 v = M[(size_t)i * ld + p];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) {
            best = a;
            bi = i;
        }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {  // ties keep the lower row (first maximal pivot)
        if (threadIdx.x < s) {
            const double o = sv[threadIdx.x + s];
            const int oi = si[threadIdx.x + s];
            if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = o;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const int r = si[0];
    if (!(sv[0] > 0.0)) {
        if (threadIdx.x == 0) bad[col] = 1;
        return;
    }
    if (r != p)
        for (int j = threadIdx.x; j < ld; j += blockDim.x) {
            const double2 t = M[(size_t)p * ld + j];
            M[(size_t)p * ld + j] = M[(size_t)r * ld + j];
            M[(size_t)r * ld + j] = t;
        }
    __syncthreads();
    const double2 piv = M[(size_t)p * ld + p];
    __syncthreads();
    for (int j = threadIdx.x; j < ld; j += blockDim.x) M[(size_t)p * ld + j] = cdiv_d(M[(size_t)p * ld + j], piv);
    __syncthreads();
    for (int i = threadIdx.x; i < q; i += blockDim.x) fac[(size_t)col * q + i] = M[(size_t)i * ld + p];
}

// A[i][j] -= fac[i] A[p][j] for every row i != p (columns j >= p on the left half carry
// the reduction; the right half is the inverse being formed).
__global__ void __launch_bounds__(256) k_gj_eliminate(double2* __restrict__ A, int q, int p,
                                                      const double2* __restrict__ fac, const int* __restrict__ bad) {
    const int col = blockIdx.y;
    if (bad[col]) return;
    double2* M = A + (size_t)col * q * 2 * q;
    const int ld = 2 * q;
    const int w = ld - p;  // columns p .. 2q-1
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)q * w) return;
    const int i = (int)(e / w);
    const int j = p + (int)(e - (int64_t)i * w);
    if (i == p) return;
    const double2 f = fac[(size_t)col * q + i];
    const double2 pr = M[(size_t)p * ld + j];
    double2 v = M[(size_t)i * ld + j];
    v.x -= f.x * pr.x - f.y * pr.y;
    v.y -= f.x * pr.y + f.y * pr.x;
    M[(size_t)i * ld + j] = v;
}

// [X | I] from X (q x q per column), and after the inversion the Newton update
// X <- (X + X^{-1}) / 2 with the per-column sums ||X_new - X||^2 and ||X_new||^2.
__global__ void k_gj_load(const double2* __restrict__ X, double2* __restrict__ A, int q) {
    const int col = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)q * 2 * q) return;
    const int i = (int)(e / (2 * q)), j = (int)(e - (int64_t)i * 2 * q);
    A[(size_t)col * q * 2 * q + e] =
        j < q ? X[(size_t)col * q * q + (size_t)i * q + j] : make_double2(j - q == i ? 1.0 : 0.0, 0.0);
}
__global__ void __launch_bounds__(256) k_newton_update(double2* __restrict__ X, const double2* __restrict__ A, int q,
                                                       double* __restrict__ sums) {
    const int col = blockIdx.x;
    __shared__ double sd[256], sx[256];
    double dn = 0, xn = 0;
    for (int64_t e = threadIdx.x; e < (int64_t)q * q; e += blockDim.x) {
        const int i = (int)(e / q), j = (int)(e - (int64_t)i * q);
        const double2 xo = X[(size_t)col * q * q + e];
        const double2 xi = A[(size_t)col * q * 2 * q + (size_t)i * 2 * q + q + j];
        const double2 xn1 = make_double2(0.5 * (xo.x + xi.x), 0.5 * (xo.y + xi.y));
        dn += (xn1.x - xo.x) * (xn1.x - xo.x) + (xn1.y - xo.y) * (xn1.y - xo.y);
        xn += xn1.x * xn1.x + xn1.y * xn1.y;
        X[(size_t)col * q * q + e] = xn1;
    }
    sd[threadIdx.x] = dn;
    sx[threadIdx.x] = xn;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sd[threadIdx.x] += sd[threadIdx.x + s];
            sx[threadIdx.x] += sx[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[2 * col] = sd[0];
        sums[2 * col + 1] = sx[0];
    }
}

// sign(X_col) for ncol matrices of size q (row-major, device) by Roberts' Newton iteration,
// every column until its update falls below 1e-12 of the iterate, then once more.  Returns
// 1 if a column met a singular iterate or did not converge in 100 steps.
int newton_sign_gpu(sgn_ctx* c, double2* X, int q, int ncol, int* failed) {
    cudaStream_t st = c->work;
    const size_t aug = (size_t)ncol * q * 2 * q;
    DevBuf buf;
    const size_t oA = 0, of = align256(sizeof(double2) * aug), ob = of + align256(sizeof(double2) * ncol * q),
                 os = ob + align256(sizeof(int) * ncol);
    SGN_CHECK(dev_alloc(c, buf, os + align256(sizeof(double) * 2 * ncol)));
    char* base = reinterpret_cast<char*>(buf.p);
    double2* A = reinterpret_cast<double2*>(base + oA);
    double2* fac = reinterpret_cast<double2*>(base + of);
    int* bad = reinterpret_cast<int*>(base + ob);
    double* sums = reinterpret_cast<double*>(base + os);
    auto done_with = [&](int rc) {
        dev_free(c, buf);
        return rc;
    };
    // one inversion = 2q launches: captured once, replayed every Newton step
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const int64_t cells = (int64_t)q * 2 * q;
        k_gj_load<<<dim3((unsigned)((cells + 255) / 256), ncol), 256, 0, st>>>(X, A, q);
        for (int p = 0; p < q && e == cudaSuccess; ++p) {
            k_gj_pivot<<<ncol, 256, 0, st>>>(A, q, p, fac, bad);
            const int64_t work = (int64_t)q * (2 * q - p);
            k_gj_eliminate<<<dim3((unsigned)((work + 255) / 256), ncol), 256, 0, st>>>(A, q, p, fac, bad);
            e = cudaGetLastError();
        }
        k_newton_update<<<ncol, 256, 0, st>>>(X, A, q, sums);
        cudaError_t ee = cudaStreamEndCapture(st, &g);
        if (e == cudaSuccess) e = ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error(std::string("apply_direct: Newton graph: ") + cudaGetErrorString(e));
        return done_with(SGN_ERR_CUDA);
    }
    // per column: 0 iterating, 1 update below 1e-12 of the iterate (one more step to take),
    // 2 finished; every column steps with the others (a converged X is a fixed point)
    std::vector<double> hs(2 * ncol);
    std::vector<int> hb(ncol), state(ncol, 0);
    bool launch_ok = cudaMemsetAsync(bad, 0, sizeof(int) * ncol, st) == cudaSuccess;
    for (int it = 0; it < 100 && launch_ok; ++it) {
        if (cudaGraphLaunch(ge, st) != cudaSuccess ||
            cudaMemcpyAsync(hs.data(), sums, sizeof(double) * 2 * ncol, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hb.data(), bad, sizeof(int) * ncol, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            launch_ok = false;
            break;
        }
        count_launch(2 + 2LL * q);
        bool all = true;
        for (int col = 0; col < ncol; ++col) {
            if (hb[col] || state[col] == 2) continue;
            if (state[col] == 1) {
                state[col] = 2;
                continue;
            }
            if (std::sqrt(hs[2 * col]) <= 1e-12 * std::sqrt(hs[2 * col + 1])) state[col] = 1;
            all = false;
        }
        if (all) break;
    }
    cudaGraphExecDestroy(ge);
    if (!launch_ok) {
        set_error("apply_direct: Newton iteration launch failed");
        return done_with(SGN_ERR_CUDA);
    }
    for (int col = 0; col < ncol; ++col)
        if (hb[col] || state[col] != 2) failed[col] = 1;
    return done_with(SGN_OK);
}

}  // namespace

int direct_projection(sgn_ctx* c, const double2* b, double2* x, int ncol, int k, bool adjoint, int* kk_out) {
    using cd = std::complex<double>;
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    const int m = c->m;
    const size_t field = (size_t)n * sizeof(double2);
    const int rs = GS_BLOCK + 8;
    const int nblk = reduce_blocks<double2>(n);
    const size_t oV = 0, ow = oV + align256(field * (size_t)(k + 1) * ncol);
    const size_t op = ow + align256(field * ncol);
    const size_t ored = op + align256(sizeof(double2) * (size_t)ncol * rs * nblk);
    const size_t ocoef = ored + align256(sizeof(double2) * (size_t)ncol * rs);
    const size_t oflag = ocoef + align256(sizeof(double2) * (size_t)ncol * rs);
    const size_t total = oflag + align256(sizeof(int) * 2 * (size_t)ncol);
    DevBuf buf;
    SGN_CHECK(dev_alloc(c, buf, total));
    char* base = reinterpret_cast<char*>(buf.p);
    double2* V = reinterpret_cast<double2*>(base + oV);
    double2* w = reinterpret_cast<double2*>(base + ow);
    double2* coef = reinterpret_cast<double2*>(base + ocoef);
    const Reduce rd{reinterpret_cast<double2*>(base + op), nblk, rs};
    DevState S{};
    S.red = reinterpret_cast<double2*>(base + ored);
    S.skip = reinterpret_cast<int*>(base + oflag);
    S.done = S.skip + ncol;
    S.rstride = rs;
    const int64_t sj = (int64_t)ncol * n;
    std::vector<double2> hbuf((size_t)ncol * rs);
    auto bail = [&](int e) {
        dev_free(c, buf);
        return e;
    };
#define DC(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            set_error(std::string("apply_direct: ") + cudaGetErrorString(e_));      \
            return bail(SGN_ERR_CUDA);                                               \
        }                                                                            \
    } while (0)
    auto fetch = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(hbuf.data(), S.red, sizeof(double2) * hbuf.size(), cudaMemcpyDeviceToHost, st);
        return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
    };
    auto upload = [&](const std::vector<cd>& C, int J, int j0) -> cudaError_t {  // C[col][j0 .. j0+J) -> coef
        std::vector<double2> h((size_t)ncol * rs, make_double2(0, 0));
        const int ld = (int)(C.size() / ncol);
        for (int col = 0; col < ncol; ++col)
            for (int j = 0; j < J; ++j) {
                const cd v = C[(size_t)col * ld + j0 + j];
                h[(size_t)col * rs + j] = make_double2(v.real(), v.imag());
            }
        cudaError_t e = cudaMemcpyAsync(coef, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, st);
        return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
    };
    DC(cudaMemsetAsync(S.skip, 0, sizeof(int) * 2 * ncol, st));
    DC(cudaMemsetAsync(x, 0, field * ncol, st));
    // x_P and r = (I - P) b (eqs. (4.2), (4.3)); r goes to w
    const double2* Lb = reinterpret_cast<const double2*>(adjoint ? c->R64.p : c->L64.p);
    const double2* Rb = reinterpret_cast<const double2*>(adjoint ? c->L64.p : c->R64.p);
    const double2* lam = reinterpret_cast<const double2*>(adjoint ? c->lamc_dev.p : c->lam_dev.p);
    if (m > 0) {
        if (m > GS_BLOCK) {
            set_error("apply_direct: deflation size above 128");
            return bail(SGN_ERR_ARG);
        }
        const Basis<double2> LB{Lb, n, 0}, RB{Rb, n, 0};
        DC(mdot<double2>(LB, m, b, n, n, ncol, rd, 0, nullptr, st));
        DC(reduce(rd, m, ncol, RM_SIGNED, 0, S, lam, st));
        DC(update_x<double2>(RB, m, S.red, rs, x, n, n, ncol, nullptr, nullptr, st));
        DC(reduce(rd, m, ncol, RM_STORE, 0, S, nullptr, st));
        DC(maxpy_scale<double2>(RB, m, S.red, rs, b, n, w, n, nullptr, n, ncol, nullptr, st));
    } else {
        DC(cudaMemcpyAsync(w, b, field * ncol, cudaMemcpyDeviceToDevice, st));
    }
    auto norms = [&](std::vector<double>& out) -> cudaError_t {  // ||w|| per column
        cudaError_t e = mdot<double2>(Basis<double2>{w, 0, n}, 0, w, n, n, ncol, rd, 1, nullptr, st);
        if (e == cudaSuccess) e = reduce(rd, 1, ncol, RM_STORE, 0, S, nullptr, st);
        if (e == cudaSuccess) e = fetch();
        for (int col = 0; col < ncol && e == cudaSuccess; ++col) out[col] = std::sqrt(std::max(hbuf[(size_t)col * rs].x, 0.0));
        return e;
    };
    auto normalize_into = [&](double2* dst, const std::vector<double>& nr) -> cudaError_t {  // dst = w / nr
        std::vector<cd> D(ncol);
        for (int col = 0; col < ncol; ++col) D[col] = nr[col] > 0 ? 1.0 / nr[col] : 0.0;
        cudaError_t e = upload(D, 1, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, field * ncol, st);
        if (e == cudaSuccess)
            e = update_x<double2>(Basis<double2>{w, 0, n}, 1, coef, rs, dst, n, n, ncol, nullptr, nullptr, st);
        return e;
    };
    std::vector<double> beta(ncol), hn(ncol);
    DC(norms(beta));
    DC(normalize_into(V, beta));
    // Arnoldi on A (eq. (2.4)); column col stops growing at its first breakdown
    std::vector<cd> H((size_t)ncol * (k + 1) * k, 0.0);
    std::vector<int> kk(ncol, k);
    std::vector<char> live(ncol);
    for (int col = 0; col < ncol; ++col) {
        live[col] = beta[col] > 0;
        if (!live[col]) kk[col] = 0;
    }
    for (int j = 0; j < k; ++j) {
        DC(apply_hw64(c, w, V + (size_t)j * sj, ncol, adjoint, nullptr, st));
        for (int pass = 0; pass < 2; ++pass)
            for (int i0 = 0; i0 <= j; i0 += GS_BLOCK) {
                const int J = std::min(GS_BLOCK, j + 1 - i0);
                const Basis<double2> VB{V + (size_t)i0 * sj, sj, n};
                DC(mdot<double2>(VB, J, w, n, n, ncol, rd, 0, nullptr, st));
                DC(reduce(rd, J, ncol, RM_STORE, 0, S, nullptr, st));
                DC(fetch());
                for (int col = 0; col < ncol; ++col)
                    for (int i = 0; i < J; ++i) {
                        const double2 h = hbuf[(size_t)col * rs + i];
                        H[((size_t)col * (k + 1) + i0 + i) * k + j] += cd(h.x, h.y);
                    }
                DC(maxpy_scale<double2>(VB, J, S.red, rs, w, n, w, n, nullptr, n, ncol, nullptr, st));
            }
        DC(norms(hn));
        for (int col = 0; col < ncol; ++col) {
            if (!live[col]) {
                hn[col] = 0;
                continue;
            }
            double cn = hn[col] * hn[col];
            for (int i = 0; i <= j; ++i) cn += std::norm(H[((size_t)col * (k + 1) + i) * k + j]);
            if (hn[col] <= 1e-14 * std::sqrt(cn)) {  // invariant subspace: the projection is exact
                live[col] = 0;
                kk[col] = j + 1;
                hn[col] = 0;
            } else {
                H[((size_t)col * (k + 1) + j + 1) * k + j] = hn[col];
            }
        }
        DC(normalize_into(V + (size_t)(j + 1) * sj, hn));
        if (std::none_of(live.begin(), live.end(), [](char v) { return v != 0; })) break;
    }
    // y_col = beta sign(H_kk) e_1: Roberts' Newton iteration for all columns on the GPU,
    // each H_kk padded to the largest Krylov dimension with the identity
    const int kmaxu = *std::max_element(kk.begin(), kk.end());
    const int qd = std::max(kmaxu, 1);
    std::vector<cd> Y((size_t)ncol * qd, 0.0);
    std::vector<int> fail(ncol, 0);
    if (kmaxu > 0) {
        std::vector<double2> Xh((size_t)ncol * qd * qd, make_double2(0, 0));
        for (int col = 0; col < ncol; ++col) {
            const int q = kk[col];
            for (int r = 0; r < qd; ++r)
                for (int l = 0; l < qd; ++l) {
                    cd v = (r < q && l < q) ? H[((size_t)col * (k + 1) + r) * k + l] : cd(r == l ? 1.0 : 0.0, 0.0);
                    Xh[((size_t)col * qd + r) * qd + l] = make_double2(v.real(), v.imag());
                }
        }
        DevBuf xb;
        const int ra = dev_alloc(c, xb, sizeof(double2) * Xh.size());
        if (ra != SGN_OK) return bail(ra);
        double2* Xd = reinterpret_cast<double2*>(xb.p);
        auto xfail = [&](int code) {
            dev_free(c, xb);
            return bail(code);
        };
        if (cudaMemcpyAsync(Xd, Xh.data(), sizeof(double2) * Xh.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("apply_direct: copying H_k to the device failed");
            return xfail(SGN_ERR_CUDA);
        }
        const int rn = newton_sign_gpu(c, Xd, qd, ncol, fail.data());
        if (rn != SGN_OK) return xfail(rn);
        if (cudaMemcpyAsync(Xh.data(), Xd, sizeof(double2) * Xh.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            set_error("apply_direct: copying sign(H_k) to the host failed");
            return xfail(SGN_ERR_CUDA);
        }
        dev_free(c, xb);
        for (int col = 0; col < ncol; ++col)
            for (int r = 0; r < kk[col]; ++r) {
                const double2 v = Xh[((size_t)col * qd + r) * qd];  // first column of sign(H)
                Y[(size_t)col * qd + r] = beta[col] * cd(v.x, v.y);
            }
    }
    if (std::any_of(fail.begin(), fail.end(), [](int f) { return f != 0; })) {
        set_error("apply_direct: Newton iteration for sign(H_k) failed (singular iterate or no convergence)");
        return bail(SGN_ERR_NOT_CONVERGED);
    }
    // x += V_k y, in blocks
    for (int i0 = 0; i0 < kmaxu; i0 += GS_BLOCK) {
        const int J = std::min(GS_BLOCK, kmaxu - i0);
        DC(upload(Y, J, i0));
        DC(update_x<double2>(Basis<double2>{V + (size_t)i0 * sj, sj, n}, J, coef, rs, x, n, n, ncol, nullptr, nullptr,
                             st));
    }
    DC(cudaStreamSynchronize(st));
#undef DC
    if (kk_out) *kk_out = kmaxu;
    dev_free(c, buf);
    return SGN_OK;
}

}  // namespace sgn
