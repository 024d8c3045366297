// Deflation set-up: critical eigenpairs of H_W(mu) on the GPU (Sec. 4).
#include "ctx.cuh"

namespace sgn {

int build_deflation(sgn_ctx* c, int m, int extra, double eig_tol, double* lambda_out) {
    (void)c;
    (void)m;
    (void)extra;
    (void)eig_tol;
    (void)lambda_out;
    set_error("sgn_build_deflation: the eigensolver is not part of this build");
    return SGN_ERR_DEFLATION;
}

}  // namespace sgn
