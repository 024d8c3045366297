// The overlap operator built on the sign function (Sec. 1: the reason sign(H_W(mu))
// is needed):  D_ov = 1 + gamma5 F(A),  F(A) the deflated rational sign function of
// Algorithm 1 that sgn_apply computes, and the solution of D_ov x = b by restarted
// GMRES whose every Arnoldi step is one batched sign solve over all columns.  The
// outer Gram-Schmidt (two classical passes), the Hessenberg least squares (Givens, on
// the host: k <= 64 per column) and the update x += V y use the library's FP64 kernels.
#include "ctx.cuh"

#include <algorithm>

namespace sgn {

// y = b + gamma5 F(A) b on ncol packed FP64 fields (y and b may not overlap)
int overlap_apply(sgn_ctx* c, const double2* b, double2* y, int ncol, sgn_report* rep) {
    cudaStream_t st = c->work;
    DevBuf buf;
    SGN_CHECK(dev_alloc(c, buf, sizeof(double2) * (size_t)c->n * ncol));
    double2* fx = reinterpret_cast<double2*>(buf.p);
    int status = solve(c, b, fx, nullptr, ncol, false, false, rep);
    if (status == SGN_OK) {
        cudaError_t e = gamma5_axpy(y, b, fx, 1.0, c->vol, ncol, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error(std::string("overlap_apply: ") + cudaGetErrorString(e));
            status = SGN_ERR_CUDA;
        }
    }
    dev_free(c, buf);
    return status;
}

// D_ov x = b by GMRES(k) restarted from x, per-column convergence ||r|| <= tol ||b||.
int overlap_solve(sgn_ctx* c, const double2* b, double2* x, int ncol, double tol, int k, int max_restarts,
                  int* iterations, double* relres) {
    using cd = std::complex<double>;
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    const size_t field = (size_t)n * sizeof(double2);
    const int rs = ((k + 2) + 7) & ~7;
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
    const Basis<double2> VB{V, sj, n};
    std::vector<double2> hbuf((size_t)ncol * rs);
    auto fetch = [&]() -> int {  // S.red -> hbuf
        SGN_CUDA(cudaMemcpyAsync(hbuf.data(), S.red, sizeof(double2) * hbuf.size(), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        return SGN_OK;
    };
    auto upload = [&](const std::vector<cd>& C, int J) -> int {  // [col][j] -> coef
        std::vector<double2> h((size_t)ncol * rs, make_double2(0, 0));
        for (int col = 0; col < ncol; ++col)
            for (int j = 0; j < J; ++j) h[(size_t)col * rs + j] = make_double2(C[(size_t)col * J + j].real(), C[(size_t)col * J + j].imag());
        SGN_CUDA(cudaMemcpyAsync(coef, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        return SGN_OK;
    };
    int status = SGN_OK;
    auto bail = [&](int e) {
        dev_free(c, buf);
        return e;
    };
#define OC(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) {                                    \
            set_error(std::string("overlap_solve: ") + cudaGetErrorString(e_)); \
            return bail(SGN_ERR_CUDA);                              \
        }                                                           \
    } while (0)
#define OR(call)                      \
    do {                              \
        int e_ = (call);              \
        if (e_ != SGN_OK) return bail(e_); \
    } while (0)
    OC(cudaMemsetAsync(S.skip, 0, sizeof(int) * 2 * ncol, st));
    // ||b|| per column
    OC(mdot<double2>(Basis<double2>{b, 0, n}, 0, b, n, n, ncol, rd, 1, nullptr, st));
    OC(reduce(rd, 1, ncol, RM_STORE, 0, S, nullptr, st));
    OR(fetch());
    std::vector<double> bnorm(ncol), rnorm(ncol);
    for (int col = 0; col < ncol; ++col) bnorm[col] = std::sqrt(hbuf[(size_t)col * rs].x);
    // r = b - D x (x given), into V[0]
    OR(overlap_apply(c, x, w, ncol, nullptr));
    OC(axpby3<double2>(V, 1.0, b, -1.0, w, 0.0, nullptr, sj, st));
    int its = 0;
    std::vector<cd> H((size_t)ncol * (k + 1) * k), g((size_t)ncol * (k + 1));
    std::vector<cd> cs((size_t)ncol * k), sn((size_t)ncol * k);
    for (int restart = 0; restart <= max_restarts; ++restart) {
        OC(mdot<double2>(Basis<double2>{V, 0, n}, 0, V, n, n, ncol, rd, 1, nullptr, st));
        OC(reduce(rd, 1, ncol, RM_STORE, 0, S, nullptr, st));
        OR(fetch());
        bool all = true;
        for (int col = 0; col < ncol; ++col) {
            rnorm[col] = std::sqrt(hbuf[(size_t)col * rs].x);
            if (rnorm[col] > tol * bnorm[col]) all = false;
        }
        if (all || restart == max_restarts) break;
        {  // v_0 = r / ||r||
            std::vector<cd> D((size_t)ncol, 0.0);
            for (int col = 0; col < ncol; ++col) D[col] = rnorm[col] > 0 ? 1.0 / rnorm[col] : 0.0;
            OR(upload(D, 1));
            OC(cudaMemsetAsync(w, 0, field * ncol, st));
            OC(update_x<double2>(Basis<double2>{V, 0, n}, 1, coef, rs, w, n, n, ncol, nullptr, nullptr, st));
            OC(cudaMemcpyAsync(V, w, field * ncol, cudaMemcpyDeviceToDevice, st));
        }
        std::fill(H.begin(), H.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        for (int col = 0; col < ncol; ++col) g[(size_t)col * (k + 1)] = rnorm[col];
        int kk = k;
        for (int j = 0; j < k; ++j) {
            // w = D v_j: one batched sign solve over the columns
            OR(overlap_apply(c, V + (size_t)j * sj, w, ncol, nullptr));
            ++its;
            // two classical Gram-Schmidt passes against v_0..v_j
            for (int pass = 0; pass < 2; ++pass) {
                OC(mdot<double2>(VB, j + 1, w, n, n, ncol, rd, 0, nullptr, st));
                OC(reduce(rd, j + 1, ncol, RM_STORE, 0, S, nullptr, st));
                OR(fetch());
                for (int col = 0; col < ncol; ++col)
                    for (int i = 0; i <= j; ++i) {
                        const double2 h = hbuf[(size_t)col * rs + i];
                        H[((size_t)col * (k + 1) + i) * k + j] += cd(h.x, h.y);
                    }
                OC(maxpy_scale<double2>(VB, j + 1, S.red, rs, w, n, w, n, nullptr, n, ncol, nullptr, st));
            }
            OC(mdot<double2>(Basis<double2>{w, 0, n}, 0, w, n, n, ncol, rd, 1, nullptr, st));
            OC(reduce(rd, 1, ncol, RM_STORE, 0, S, nullptr, st));
            OR(fetch());
            std::vector<cd> D((size_t)ncol, 0.0);
            bool conv = true;
            for (int col = 0; col < ncol; ++col) {
                const double hn = std::sqrt(std::max(hbuf[(size_t)col * rs].x, 0.0));
                H[((size_t)col * (k + 1) + j + 1) * k + j] = hn;
                D[col] = hn > 0 ? 1.0 / hn : 0.0;
                // Givens on column j of this column's Hessenberg, the running residual |g_{j+1}|
                cd* Hc = &H[(size_t)col * (k + 1) * k];
                cd* gc = &g[(size_t)col * (k + 1)];
                for (int i = 0; i < j; ++i) {
                    const cd a = Hc[i * k + j], bb = Hc[(i + 1) * k + j];
                    Hc[i * k + j] = std::conj(cs[(size_t)col * k + i]) * a + std::conj(sn[(size_t)col * k + i]) * bb;
                    Hc[(i + 1) * k + j] = -sn[(size_t)col * k + i] * a + cs[(size_t)col * k + i] * bb;
                }
                const cd a = Hc[j * k + j], bb = Hc[(j + 1) * k + j];
                const double nr = std::sqrt(std::norm(a) + std::norm(bb));
                const cd cc = nr > 0 ? a / nr : cd(1.0), ss = nr > 0 ? bb / nr : cd(0.0);
                cs[(size_t)col * k + j] = cc;
                sn[(size_t)col * k + j] = ss;
                Hc[j * k + j] = std::conj(cc) * a + std::conj(ss) * bb;
                Hc[(j + 1) * k + j] = 0.0;
                const cd g0 = gc[j];
                gc[j] = std::conj(cc) * g0;
                gc[j + 1] = -ss * g0;
                if (std::abs(gc[j + 1]) > tol * bnorm[col]) conv = false;
            }
            OR(upload(D, 1));
            OC(cudaMemsetAsync(V + (size_t)(j + 1) * sj, 0, field * ncol, st));
            OC(update_x<double2>(Basis<double2>{w, 0, n}, 1, coef, rs, V + (size_t)(j + 1) * sj, n, n, ncol, nullptr,
                                 nullptr, st));
            if (conv) {
                kk = j + 1;
                break;
            }
        }
        // y = R^{-1} g per column; x += V y; r = b - D x recomputed at the next restart's top
        std::vector<cd> Y((size_t)ncol * kk, 0.0);
        for (int col = 0; col < ncol; ++col) {
            const cd* Hc = &H[(size_t)col * (k + 1) * k];
            const cd* gc = &g[(size_t)col * (k + 1)];
            for (int i = kk - 1; i >= 0; --i) {
                cd z = gc[i];
                for (int l = i + 1; l < kk; ++l) z -= Hc[i * k + l] * Y[(size_t)col * kk + l];
                Y[(size_t)col * kk + i] = Hc[i * k + i] != 0.0 ? z / Hc[i * k + i] : 0.0;
            }
        }
        OR(upload(Y, kk));
        OC(update_x<double2>(VB, kk, coef, rs, x, n, n, ncol, nullptr, nullptr, st));
        // true residual for the restart: r = b - D x
        OR(overlap_apply(c, x, w, ncol, nullptr));
        OC(axpby3<double2>(V, 1.0, b, -1.0, w, 0.0, nullptr, sj, st));
    }
#undef OC
#undef OR
    double worst = 0;
    for (int col = 0; col < ncol; ++col) worst = std::max(worst, bnorm[col] > 0 ? rnorm[col] / bnorm[col] : 0.0);
    if (iterations) *iterations = its;
    if (relres) *relres = worst;
    if (worst > tol) {
        set_error("overlap_solve: max_restarts reached before every column met the tolerance");
        status = SGN_ERR_NOT_CONVERGED;
    }
    dev_free(c, buf);
    return status;
}

}  // namespace sgn
