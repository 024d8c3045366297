// The direct projection that the paper compares Algorithm 1 against (Sec. 6, eq. (6.3)):
//   x = x_P + ||r|| V_k sign(H_k) e_1,   r = (I - P) b,   x_P = R sign(Re Lambda) L^dag b,
// with V_k, H_k from k Arnoldi steps on A itself (no rational approximation, no restarts),
// and sign(H_k) by Roberts' Newton iteration X <- (X + X^{-1}) / 2 on the k x k matrix.
// The whole basis is kept (k + 1 FP64 fields per column, the method's memory cost); the
// Arnoldi steps use the FP64 stencil and two classical Gram-Schmidt passes, in blocks of at
// most 128 basis vectors per kernel (the reduction's slot limit).  The k x k Newton
// iterations run on the host, one thread per column.
#include "ctx.cuh"
#include "dense_eig.h"

#include <algorithm>
#include <thread>

namespace sgn {

namespace {
constexpr int GS_BLOCK = 128;

// sign(M) of a small dense matrix (row-major kk x kk) by Roberts' Newton iteration:
// iterate until the update falls below 1e-12 of the iterate, then once more (quadratic
// convergence takes that step to rounding level).  Returns 0, or 1 on a singular iterate
// or no convergence in 100 steps.
int roberts_sign(int kk, std::vector<std::complex<double>>& X) {
    using cd = std::complex<double>;
    int extra = -1;
    for (int it = 0; it < 100; ++it) {
        std::vector<cd> inv((size_t)kk * kk, 0.0);
        for (int i = 0; i < kk; ++i) inv[(size_t)i * kk + i] = 1.0;
        if (dense_solve(kk, kk, X, inv)) return 1;
        double dn = 0, xn = 0;
        for (size_t e = 0; e < X.size(); ++e) {
            const cd xn1 = 0.5 * (X[e] + inv[e]);
            dn += std::norm(xn1 - X[e]);
            xn += std::norm(xn1);
            X[e] = xn1;
        }
        if (extra == 0) return 0;
        if (extra < 0 && std::sqrt(dn) <= 1e-12 * std::sqrt(xn)) extra = 0;
    }
    return 1;
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
    // y_col = beta sign(H_kk) e_1, on the host, one thread per column
    const int kmaxu = *std::max_element(kk.begin(), kk.end());
    std::vector<cd> Y((size_t)ncol * std::max(kmaxu, 1), 0.0);
    std::vector<int> fail(ncol, 0);
    auto work = [&](int col) {
        const int q = kk[col];
        if (q == 0) return;
        std::vector<cd> X((size_t)q * q);
        for (int r = 0; r < q; ++r)
            for (int l = 0; l < q; ++l) X[(size_t)r * q + l] = H[((size_t)col * (k + 1) + r) * k + l];
        fail[col] = roberts_sign(q, X);
        for (int r = 0; r < q; ++r) Y[(size_t)col * std::max(kmaxu, 1) + r] = beta[col] * X[(size_t)r * q];
    };
    {
        const int nt = std::max(1, std::min<int>(ncol, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        bool serial = false;
        try {
            for (int t = 1; t < nt; ++t)
                pool.emplace_back([&, t]() {
                    for (int col = t; col < ncol; col += nt) work(col);
                });
        } catch (...) {  // a thread could not be started: every column runs here (work is idempotent)
            serial = true;
        }
        if (!serial)
            for (int col = 0; col < ncol; col += nt) work(col);
        for (auto& th : pool) th.join();
        if (serial)
            for (int col = 0; col < ncol; ++col) work(col);
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
