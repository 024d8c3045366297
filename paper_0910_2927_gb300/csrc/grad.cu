// Derivative of x = sum_i omega_i A (A^2 - sigma_i)^{-1} b with respect to mu
// (the undeflated rational function of eq. (6.2), A = H_W(mu)).  With
// A' = dA/dmu and x_i = (A^2 - sigma_i)^{-1} A b,
//   d/dmu [A (A^2 - sigma)^{-1}] b = (A^2 - sigma)^{-1} [A' b - (A' A + A A') x_i],
// so for a loss Re<g, x>:  dmu = Re sum_i omega_i <z_i, A' b - A' A x_i - A A' x_i>
// with z_i = (A^dag^2 - sigma_i)^{-1} g, the per-shift iterates of one adjoint
// multishift solve (H_W(mu)^dag = H_W(-mu)).
#include "ctx.cuh"

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

int grad_mu(sgn_ctx* c, const double2* b, const double2* g, int ncol, double* dmu) {
    cudaStream_t st = c->work;
    const int s = (int)c->sigma.size();
    const int64_t n = c->n;
    const size_t field = (size_t)n * sizeof(double2);
    DevBuf buf;
    const size_t fs = ((field * ncol * s) + 255) & ~size_t(255);
    const size_t fc = ((field * ncol) + 255) & ~size_t(255);
    SGN_CHECK(dev_alloc(c, buf, 2 * fs + 5 * fc));
    char* p = reinterpret_cast<char*>(buf.p);
    double2* xs = reinterpret_cast<double2*>(p);
    double2* zs = reinterpret_cast<double2*>(p + fs);
    double2* x = reinterpret_cast<double2*>(p + 2 * fs);
    double2* apb = reinterpret_cast<double2*>(p + 2 * fs + fc);
    double2* t1 = reinterpret_cast<double2*>(p + 2 * fs + 2 * fc);
    double2* t2 = reinterpret_cast<double2*>(p + 2 * fs + 3 * fc);
    double2* r = reinterpret_cast<double2*>(p + 2 * fs + 4 * fc);
    int rc = solve(c, b, x, xs, ncol, false, false, nullptr);
    if (rc == SGN_OK) rc = solve(c, g, x, zs, ncol, true, true, nullptr);
    if (rc != SGN_OK) {
        dev_free(c, buf);
        return rc;
    }
    std::vector<double> acc(ncol, 0.0);
    SGN_CUDA(apply_dhw_dmu64(c, apb, b, ncol, st));
    for (int i = 0; i < s; ++i) {
        const double2* xi = xs + (size_t)i * ncol * n;
        const double2* zi = zs + (size_t)i * ncol * n;
        SGN_CUDA(apply_hw64(c, t1, xi, ncol, false, nullptr, st));   // A x_i
        SGN_CUDA(apply_dhw_dmu64(c, t2, t1, ncol, st));               // A' A x_i
        SGN_CUDA(apply_dhw_dmu64(c, t1, xi, ncol, st));               // A' x_i
        SGN_CUDA(apply_hw64(c, r, t1, ncol, false, nullptr, st));    // A A' x_i
        SGN_CUDA(axpby3<double2>(r, 1.0, apb, -1.0, t2, -1.0, r, (int64_t)ncol * n, st));
        std::vector<std::complex<double>> d;
        rc = field_dots(c, zi, r, ncol, d);
        if (rc != SGN_OK) {
            dev_free(c, buf);
            return rc;
        }
        for (int col = 0; col < ncol; ++col) acc[col] += c->omega[i] * d[col].real();
    }
    SGN_CUDA(cudaStreamSynchronize(st));
    dev_free(c, buf);
    for (int col = 0; col < ncol; ++col) dmu[col] = acc[col];
    return SGN_OK;
}

}  // namespace sgn
