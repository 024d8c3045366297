// Derivative with respect to mu of the deflated rational sign function of
// Sec. 4 and eq. (6.2), A = H_W(mu):
//   x = F(A) b,  F(A) = R S L^dag + G(A) (I - P),  G(A) = sum_i omega_i (A^2 - sigma_i)^{-1} A,
// with S = diag(sign(Re lambda_j)) and P = R L^dag over the m deflated pairs.
// For a loss Re<q, x> (q = dloss/dx) and A' = dA/dmu:
//   dx = dG[A'] (I - P) b - G(A) dP b + R S dL^dag b + dR S L^dag b,
// and with the reduced resolvents S_j = (A - lambda_j)^{-1} (I - P_j), P_j = r_j l_j^dag,
// dr_j = -S_j A' r_j, dl_j^dag = -l_j^dag A' S_j (so dP_j = -S_j A' P_j - P_j A' S_j):
//   <q, dx> = A + B + C,
//   A = sum_i omega_i <z_i, A' v - A' A x_i - A A' x_i>,  v = (I - P) b,
//       x_i = (A^2 - sigma_i)^{-1} A v,  z_i = (A^dag^2 - sigma_i)^{-1} q,
//   B = -sum_j (l_j^dag b) <S_j^dag (s_j q - h), A' r_j>,  h = G(A)^dag q = G(A^dag) q,
//   C = -sum_j (s_j - g(lambda_j)) <q, r_j> l_j^dag A' S_j b,   g(t) = sum_i omega_i t / (t^2 - sigma_i).
// The reduced resolvents act through A^2:  (A - lambda)^{-1} = (A + lambda)(A^2 - lambda^2)^{-1}
// on range(I - P), where one multishift solve with the m complex shifts lambda_j^2 serves
// every j; the deflated directions k != j are exact:  (A - lambda_j)^{-1} r_k = r_k / (lambda_k - lambda_j).
// The sums over k != j run over the m deflated pairs and the mx extra pairs the
// context keeps (the next eigenpairs, not deflated in the solve); the iterative part
// then projects all m + mx of them out, so the shifts lambda_j^2 stay away from the
// spectrum it works on (with lambda_j^2 next to lambda_{m+1}^2 the system is nearly
// singular and restarted GMRES stagnates).  With m = 0 only A remains (the
// undeflated function).
#include "ctx.cuh"

#include <algorithm>

namespace sgn {

cudaError_t apply_dhw_dmu64(const sgn_ctx* c, double2* out, const double2* in, int ncol, cudaStream_t st) {
    StencilParams p = stencil_params(c, false);
    p.diag = 0.0;
    for (int d = 0; d < 3; ++d) {
        p.cf[d] = 0.0;
        p.cb[d] = 0.0;
    }
    p.cf[3] = -0.5 * std::exp(c->mu);  // d/dmu of -1/2 e^{+mu}
    p.cb[3] = 0.5 * std::exp(-c->mu);  // d/dmu of -1/2 e^{-mu}
    fill_fp32_coefficients(p);
    return launch_hw_f64(out, in, reinterpret_cast<const double2*>(c->U64.p), ncol, p, nullptr, st);
}

namespace {

using cd = std::complex<double>;

// Inner products and combinations with a small set of fields X (nx <= 64), FP64.
struct Small {
    sgn_ctx* c;
    DevBuf buf;
    Reduce rd{};
    DevState S{};
    double2* coef = nullptr;
    int rs = 0, ncap = 0;
    int init(sgn_ctx* c_, int nx, int ncols) {
        c = c_;
        rs = ((nx + 1) + 7) & ~7;
        ncap = ncols;
        const int nblk = reduce_blocks<double2>(c->n);
        const size_t pb = align256(sizeof(double2) * (size_t)ncols * rs * nblk);
        const size_t rb = align256(sizeof(double2) * (size_t)ncols * rs);
        const size_t fb = align256(sizeof(int) * 2 * (size_t)ncols);
        SGN_CHECK(dev_alloc(c, buf, pb + 2 * rb + fb));
        char* p = reinterpret_cast<char*>(buf.p);
        rd = Reduce{reinterpret_cast<double2*>(p), nblk, rs};
        S.red = reinterpret_cast<double2*>(p + pb);
        coef = reinterpret_cast<double2*>(p + pb + rb);
        S.skip = reinterpret_cast<int*>(p + pb + 2 * rb);
        S.done = S.skip + ncols;
        S.rstride = rs;
        SGN_CUDA(cudaMemsetAsync(S.skip, 0, sizeof(int) * 2 * ncols, c->work));
        return SGN_OK;
    }
    void release() { dev_free(c, buf); }
    // G[col][j] = <X_j, Y_col>  (X: nx fields, Y: ny fields)
    int gram(const double2* X, int nx, const double2* Y, int ny, std::vector<cd>& G) {
        const int64_t n = c->n;
        cudaStream_t st = c->work;
        if (ny > ncap || nx + 1 > rs) {
            set_error("gradient: internal size");
            return SGN_ERR_ARG;
        }
        SGN_CUDA(mdot<double2>(Basis<double2>{X, n, 0}, nx, Y, n, n, ny, rd, 0, nullptr, st));
        SGN_CUDA(reduce(rd, nx, ny, RM_STORE, 0, S, nullptr, st));
        std::vector<double2> h((size_t)ny * rs);
        SGN_CUDA(cudaMemcpyAsync(h.data(), S.red, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        G.assign((size_t)ny * nx, 0.0);
        for (int col = 0; col < ny; ++col)
            for (int j = 0; j < nx; ++j) G[(size_t)col * nx + j] = {h[(size_t)col * rs + j].x, h[(size_t)col * rs + j].y};
        return SGN_OK;
    }
    // Y_col += sum_j X_j C[col][j]
    int combine(const double2* X, int nx, const std::vector<cd>& C, double2* Y, int ny) {
        const int64_t n = c->n;
        cudaStream_t st = c->work;
        if (ny > ncap || nx + 1 > rs) {
            set_error("gradient: internal size");
            return SGN_ERR_ARG;
        }
        std::vector<double2> h((size_t)ny * rs, make_double2(0, 0));
        for (int col = 0; col < ny; ++col)
            for (int j = 0; j < nx; ++j)
                h[(size_t)col * rs + j] = make_double2(C[(size_t)col * nx + j].real(), C[(size_t)col * nx + j].imag());
        SGN_CUDA(cudaMemcpyAsync(coef, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, st));
        SGN_CUDA(update_x<double2>(Basis<double2>{X, n, 0}, nx, coef, rs, Y, n, n, ny, nullptr, nullptr, st));
        SGN_CUDA(cudaStreamSynchronize(st));  // h is released on return
        return SGN_OK;
    }
};

}  // namespace

int grad_mu(sgn_ctx* c, const double2* b, const double2* q, int ncol, double* dmu) {
    cudaStream_t st = c->work;
    const int s = (int)c->sigma.size();
    const int m = c->m;
    const int64_t n = c->n;
    const size_t field = (size_t)n * sizeof(double2);
    auto fields = [&](size_t cnt) { return align256(field * cnt); };
    // x_i, z_i (s ncol each) | x, v, apv, t1, t2, r, h (ncol each) | W = [q | h] (2 ncol)
    // | complex-shift iterates: adjoint (m x 2 ncol), forward (m x ncol) | A' r_j, p_j (m each)
    // | A' A y', A' y' (m ncol each)
    const size_t o_xs = 0, o_zs = o_xs + fields((size_t)s * ncol);
    size_t off = o_zs + fields((size_t)s * ncol);
    size_t o_col[7];
    for (int i = 0; i < 7; ++i) {
        o_col[i] = off;
        off += fields(ncol);
    }
    const size_t o_w = off;  // output of the (j, w) systems
    off += fields((size_t)m * 2 * ncol + 2 * (size_t)ncol);
    const size_t o_ya = off;
    off += fields((size_t)m * 2 * ncol);
    const size_t o_yf = off;
    off += fields((size_t)m * ncol);
    const int me = m + (m > 0 ? c->mx : 0);  // deflated + extra pairs for the reduced resolvents
    const size_t o_ar = off;
    off += fields(me);
    const size_t o_re = off;
    off += fields(me);
    const size_t o_le = off;
    off += fields(me);
    const size_t o_p = off;
    off += fields(m);
    const size_t o_t1 = off;
    off += fields((size_t)m * ncol);
    const size_t o_t2 = off;
    off += fields((size_t)m * ncol);
    DevBuf buf;
    SGN_CHECK(dev_alloc(c, buf, off));
    char* base = reinterpret_cast<char*>(buf.p);
    auto F = [&](size_t o) { return reinterpret_cast<double2*>(base + o); };
    double2 *xs = F(o_xs), *zs = F(o_zs), *x = F(o_col[0]), *v = F(o_col[1]), *apv = F(o_col[2]);
    double2 *t1 = F(o_col[3]), *t2 = F(o_col[4]), *r = F(o_col[5]), *h = F(o_col[6]);
    double2 *W = F(o_w), *ya = F(o_ya), *yf = F(o_yf), *Ar = F(o_ar), *pj = F(o_p), *T1 = F(o_t1), *T2 = F(o_t2);
    double2 *Re = F(o_re), *Le = F(o_le);
    Small sm;
    int rc = sm.init(c, std::max(me, 1), std::max({2 * ncol, 2 * m * ncol, me, 1}));
    auto done = [&](int status) {
        sm.release();
        dev_free(c, buf);
        return status;
    };
    if (rc != SGN_OK) return done(rc);
#define GR(call)                                \
    do {                                        \
        int e_ = (call);                        \
        if (e_ != SGN_OK) return done(e_);      \
    } while (0)
#define GC(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            set_error(std::string("gradient: ") + cudaGetErrorString(e_)); \
            return done(SGN_ERR_CUDA);                        \
        }                                                     \
    } while (0)

    const double2* R = reinterpret_cast<const double2*>(c->R64.p);
    const double2* L = reinterpret_cast<const double2*>(c->L64.p);
    std::vector<cd> lam(c->lam.begin(), c->lam.end());
    if (m > 0) lam.insert(lam.end(), c->lamx.begin(), c->lamx.begin() + (me - m));  // lam[m..me): extra pairs
    std::vector<double> sg(m);
    for (int j = 0; j < m; ++j) sg[j] = lam[j].real() > 0 ? 1.0 : -1.0;
    auto gfun = [&](cd t) {
        cd a = 0;
        for (int i = 0; i < s; ++i) a += c->omega[i] * t / (t * t - c->sigma[i]);
        return a;
    };

    // ---- A: per-shift forward iterates on v = (I - P) b and adjoint iterates on q
    GR(solve(c, b, x, xs, ncol, false, false, nullptr));
    GR(solve(c, q, x, zs, ncol, true, true, nullptr));
    std::vector<cd> cL, cR;  // [col][j]: <l_j, b>, <r_j, q>
    GC(cudaMemcpyAsync(v, b, field * ncol, cudaMemcpyDeviceToDevice, st));
    if (m > 0) {
        GR(sm.gram(L, m, b, ncol, cL));
        GR(sm.gram(R, m, q, ncol, cR));
        std::vector<cd> C((size_t)ncol * m);
        for (size_t t = 0; t < C.size(); ++t) C[t] = -cL[t];
        GR(sm.combine(R, m, C, v, ncol));  // v = b - R L^dag b
        // z_i += L (conj(Lambda)^2 - sigma_i)^{-1} R^dag q: the deflated directions of the adjoint solve
        for (int i = 0; i < s; ++i) {
            for (int col = 0; col < ncol; ++col)
                for (int j = 0; j < m; ++j) {
                    const cd lb = std::conj(lam[j]);
                    C[(size_t)col * m + j] = cR[(size_t)col * m + j] / (lb * lb - c->sigma[i]);
                }
            GR(sm.combine(L, m, C, zs + (size_t)i * ncol * n, ncol));
        }
    }
    GC(apply_dhw_dmu64(c, apv, v, ncol, st));
    std::vector<cd> total(ncol, 0.0);
    for (int i = 0; i < s; ++i) {
        const double2* xi = xs + (size_t)i * ncol * n;
        const double2* zi = zs + (size_t)i * ncol * n;
        GC(apply_hw64(c, t1, xi, ncol, false, nullptr, st));  // A x_i
        GC(apply_dhw_dmu64(c, t2, t1, ncol, st));            // A' A x_i
        GC(apply_dhw_dmu64(c, t1, xi, ncol, st));            // A' x_i
        GC(apply_hw64(c, r, t1, ncol, false, nullptr, st));   // A A' x_i
        GC(axpby3<double2>(r, 1.0, apv, -1.0, t2, -1.0, r, (int64_t)ncol * n, st));
        std::vector<cd> d;
        GR(field_dots(c, zi, r, ncol, d));
        for (int col = 0; col < ncol; ++col) total[col] += c->omega[i] * d[col];
    }

    if (m > 0) {
        // the m + mx pairs side by side
        GC(cudaMemcpyAsync(Re, R, field * m, cudaMemcpyDeviceToDevice, st));
        GC(cudaMemcpyAsync(Le, L, field * m, cudaMemcpyDeviceToDevice, st));
        if (me > m) {
            GC(cudaMemcpyAsync(Re + (size_t)m * n, c->Rx64.p, field * (me - m), cudaMemcpyDeviceToDevice, st));
            GC(cudaMemcpyAsync(Le + (size_t)m * n, c->Lx64.p, field * (me - m), cudaMemcpyDeviceToDevice, st));
        }
        // ---- h = G(A^dag) q from the adjoint apply:  x = L S R^dag q + G(A^dag)(I - P^dag) q
        GR(solve(c, q, h, nullptr, ncol, true, false, nullptr));
        {
            std::vector<cd> C((size_t)ncol * m);
            for (int col = 0; col < ncol; ++col)
                for (int j = 0; j < m; ++j)
                    C[(size_t)col * m + j] = (gfun(std::conj(lam[j])) - sg[j]) * cR[(size_t)col * m + j];
            GR(sm.combine(L, m, C, h, ncol));
        }
        std::vector<cd> cLe, cRe, cRhe;  // [col][k], k < me
        GR(sm.gram(Le, me, b, ncol, cLe));
        GR(sm.gram(Re, me, q, ncol, cRe));
        GR(sm.gram(Re, me, h, ncol, cRhe));
        // A' r_k (k < me), p_j = (A + lambda_j) A' r_j (j < m), M[k][i] = <l_i, A' r_k>
        GC(apply_dhw_dmu64(c, Ar, Re, me, st));
        GC(apply_hw64(c, pj, Ar, m, false, nullptr, st));
        {
            std::vector<cd> D((size_t)m * me, 0.0);
            for (int j = 0; j < m; ++j) D[(size_t)j * me + j] = lam[j];
            GR(sm.combine(Ar, me, D, pj, m));
        }
        std::vector<cd> M;
        GR(sm.gram(Le, me, Ar, me, M));
        // ---- B: y_j(w) = (A^dag^2 - conj(lambda_j)^2)^{-1} (I - P_e^dag) w for w = q and h, one
        // system per (j, w): the shifts lie just below the remaining spectrum, inside the
        // field of values of the non-normal A^2, so minimal-residual restarts (GMRES)
        // rather than FOM's Galerkin solves (whose H_k - shift can be singular there)
        std::vector<cd> shifts((size_t)m * 2 * ncol);
        for (int j = 0; j < m; ++j) {
            GC(cudaMemcpyAsync(ya + (size_t)j * 2 * ncol * n, q, field * ncol, cudaMemcpyDeviceToDevice, st));
            GC(cudaMemcpyAsync(ya + ((size_t)j * 2 * ncol + ncol) * n, h, field * ncol, cudaMemcpyDeviceToDevice, st));
            for (int c2 = 0; c2 < 2 * ncol; ++c2) shifts[(size_t)j * 2 * ncol + c2] = std::conj(lam[j] * lam[j]);
        }
        GR(solve_columns_gmres(c, ya, m * 2 * ncol, shifts, true, W, Re, Le, me));
        GC(cudaMemcpyAsync(ya, W, field * (size_t)m * 2 * ncol, cudaMemcpyDeviceToDevice, st));
        std::vector<cd> Py;  // [(j, col')][k] = <p_k, y_j(w_col')>
        GR(sm.gram(pj, m, ya, m * 2 * ncol, Py));
        for (int col = 0; col < ncol; ++col) {
            cd tb = 0;
            for (int j = 0; j < m; ++j) {
                const cd yq_p = std::conj(Py[((size_t)j * 2 * ncol + col) * m + j]);         // <y_j(q), p_j>
                const cd yh_p = std::conj(Py[((size_t)j * 2 * ncol + ncol + col) * m + j]);  // <y_j(h), p_j>
                cd u = sg[j] * yq_p - yh_p;
                for (int k = 0; k < me; ++k) {
                    if (k == j) continue;
                    // conj(r_k^dag w_j) / (lambda_k - lambda_j) <l_k, A' r_j>
                    const cd rkw = sg[j] * cRe[(size_t)col * me + k] - cRhe[(size_t)col * me + k];
                    u += std::conj(rkw) / (lam[k] - lam[j]) * M[(size_t)j * me + k];
                }
                tb -= cLe[(size_t)col * me + j] * u;
            }
            total[col] += tb;
        }
        // ---- C: y'_j = (A^2 - lambda_j^2)^{-1} (I - P_e) b;  l_j^dag A' S_j b
        shifts.assign((size_t)m * ncol, 0.0);
        for (int j = 0; j < m; ++j) {
            GC(cudaMemcpyAsync(T1 + (size_t)j * ncol * n, b, field * ncol, cudaMemcpyDeviceToDevice, st));
            for (int col = 0; col < ncol; ++col) shifts[(size_t)j * ncol + col] = lam[j] * lam[j];
        }
        GR(solve_columns_gmres(c, T1, m * ncol, shifts, false, yf, Re, Le, me));
        GC(apply_hw64(c, T2, yf, m * ncol, false, nullptr, st));    // A y'
        GC(apply_dhw_dmu64(c, T1, T2, m * ncol, st));              // A' A y'
        GC(apply_dhw_dmu64(c, T2, yf, m * ncol, st));              // A' y'
        std::vector<cd> E1, E2;  // [(j, col)][k] = <l_k, .>
        GR(sm.gram(Le, me, T1, m * ncol, E1));
        GR(sm.gram(Le, me, T2, m * ncol, E2));
        for (int col = 0; col < ncol; ++col) {
            cd tc = 0;
            for (int j = 0; j < m; ++j) {
                const size_t rj = ((size_t)j * ncol + col) * me + j;
                cd e = E1[rj] + lam[j] * E2[rj];  // <l_j, A' (A + lambda_j) y'_j>
                for (int k = 0; k < me; ++k) {
                    if (k == j) continue;
                    e += cLe[(size_t)col * me + k] / (lam[k] - lam[j]) * M[(size_t)k * me + j];  // <l_j, A' r_k>
                }
                const cd qr = std::conj(cR[(size_t)col * m + j]);  // <q, r_j>
                tc -= (sg[j] - gfun(lam[j])) * qr * e;
            }
            total[col] += tc;
        }
    }
#undef GR
#undef GC
    for (int col = 0; col < ncol; ++col) dmu[col] = total[col].real();
    return done(SGN_OK);
}

}  // namespace sgn
