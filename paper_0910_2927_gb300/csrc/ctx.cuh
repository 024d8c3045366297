// The context behind the opaque sgn_ctx handle and its device arena.
#pragma once

#include "blas.cuh"

#include <cmath>
#include <complex>
#include <map>
#include <memory>

struct sgn_ctx;

namespace sgn {

// A device allocation obtained through the caller's allocator (or cudaMalloc).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

int dev_alloc(sgn_ctx* c, DevBuf& b, size_t bytes);
void dev_free(sgn_ctx* c, DevBuf& b);

template <class T>
inline T* as(DevBuf& b) {
    return reinterpret_cast<T*>(b.p);
}

// Sub-buffer offsets within one allocation are rounded up to 256 bytes.
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Workspace of one FOM-LR engine configuration (columns, restart length,
// number of shifts, storage precision).  Carved out of one allocation.
struct Engine {
    int ncol = 0, k = 0, s = 0, prec = -1, m = 0;
    int64_t n = 0;
    int nblk = 0, rstride = 0;
    DevBuf arena;
    void* V = nullptr;  // (k+1) * ncol * n elements of the storage type
    void* w = nullptr;  // ncol * n
    void* t = nullptr;  // ncol * n
    double2* partial = nullptr;
    DevState S{};
    double* sigma_dev = nullptr;  // [ncol][s]
    double* omega_dev = nullptr;
    double* sigma_im_dev = nullptr;  // [ncol][s] imaginary parts (zero unless complex shifts are set)
    double* neg1 = nullptr;          // [ncol] -1.0 (scale of the FP32 minimal-residual restart vector)
    // host mirrors of the per-column flags (pinned)
    int* h_done = nullptr;
    double* h_resest = nullptr;
    int* h_err = nullptr;
    int* h_kk = nullptr;
    // captured restart cycle
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_key = 0;
    long long graph_kernels = 0;  // kernel nodes of the captured cycle
    // the whole restart loop on the device: a conditional WHILE node whose body is one
    // captured cycle and the decision kernel (k_loop_decide)
    cudaGraphExec_t loop = nullptr;
    uint64_t loop_key = 0;
    bool loop_unavailable = false;  // the runtime refused the conditional node: host loop
    int* cyc_dev = nullptr;         // [1] cycles run by the device loop
    // kernel timing: event pairs recorded inside the cycle (class, algorithmic bytes)
    std::vector<cudaEvent_t> tev;
    std::vector<std::pair<int, double>> tmarks;
};

}  // namespace sgn

struct sgn_ctx {
    int dims[4] = {0, 0, 0, 0};
    int64_t vol = 0, n = 0;
    int ap[4] = {0, 0, 0, 1};
    double mu = 0.0, mass = -1.6;
    cudaStream_t user_stream = nullptr;
    cudaStream_t work = nullptr;  // internal stream (capturable); ordered against user_stream by events
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;  // autotuner timing
    sgn_alloc_fn alloc = nullptr;
    sgn_free_fn free_ = nullptr;
    void* user = nullptr;
    int device = 0;

    // gauge field: FP64 master copy, FP32 and BF16 copies for the FP32 stencil
    sgn::DevBuf U64, U32, U16, UH, Uff;  // links: FP64, FP32, BF16, FP16, float-float (float4)
    bool have_gauge = false;

    // rational function
    std::vector<double> sigma, omega;
    // restart parameters
    int k = 40;
    double tol = 1e-10;
    int max_cycles = 1000;
    int project = 1;
    // precision
    int precision = SGN_PREC_FP64;
    double target = 1e-8;
    int link_storage = SGN_LINKS_FP32;
    int form = SGN_FORM_A2;  // Krylov space of the partial fractions (sgn_formulation)
    int method = SGN_METHOD_FOM;  // multishift FOM-LR or GMRES-LR (sgn_method)
    int k_refine = 0;    // restart length of the mixed form's correction solves (0: min(k, 16))
    int refine_batch = 0;  // shifted systems per correction batch (0: min(s nrhs, 4 nrhs), memory-bounded)

    // deflation (R, L as n x m column blocks)
    int m = 0;
    // set when a change of the operator (gauge field, mu, m_W, boundary) dropped
    // deflation data: the solves refuse (SGN_ERR_STATE) until deflation is set,
    // built or explicitly cleared (m = 0) again
    bool deflation_stale = false;
    sgn::DevBuf R64, L64, R32, L32, lam_dev, lamc_dev;
    std::vector<std::complex<double>> lam;
    // the next mx eigenpairs beyond the deflated ones (biorthonormal to them): not
    // deflated in the solve, but the derivative's reduced resolvents treat them exactly
    int mx = 0;
    sgn::DevBuf Rx64, Lx64;
    std::vector<std::complex<double>> lamx;

    // engines keyed by configuration
    std::map<uint64_t, std::unique_ptr<sgn::Engine>> engines;
    // engine of the last FP64-form multishift solve (sgn_get_hessenberg reads its H_k)
    sgn::Engine* last_fp64 = nullptr;
    // scratch fields for apply (b copy, x accumulators, FP64 temporaries)
    sgn::DevBuf io;
    sgn::DevBuf stage;  // device staging of host b / x
    sgn::DevBuf ip_scratch;  // partial sums of sgn_inner_products
    size_t io_bytes = 0;
    double2* h_pinned = nullptr;
    size_t h_pinned_bytes = 0;
    // tuned stencil launch shapes, keyed by precision * 4096 + columns
    std::map<int, sgn::StencilShape> shapes;
    // kernel timing totals per class (stencil, Gram-Schmidt reduction, Gram-Schmidt update)
    int timing = 0;
    static constexpr int kTimedClasses = 5;
    double t_ms[kTimedClasses] = {};
    long long t_launches[kTimedClasses] = {};
    double t_bytes[kTimedClasses] = {};
};

namespace sgn {

StencilParams stencil_params(const sgn_ctx* c, bool adjoint);
void fill_fp32_coefficients(StencilParams& p);
// H_W applied in FP64 / FP32 to ncol fields (skip may be null).
cudaError_t apply_hw64(const sgn_ctx* c, double2* out, const double2* in, int ncol, bool adjoint, const int* skip,
                       cudaStream_t st);
cudaError_t apply_hw32(const sgn_ctx* c, float2* out, const float2* in, int ncol, bool adjoint, const int* skip,
                       cudaStream_t st,
                       bool fp32_links = false);

int solve(sgn_ctx* c, const double2* b, double2* x, double2* x_shift, int ncol, bool adjoint, bool no_a,
          sgn_report* rep,
          const std::vector<std::complex<double>>* cshift = nullptr);
// Tuning key of the FP32 stencil for the context's link storage: 1 FP32, 2 BF16, 3 FP16 links
// (0 is the FP64 stencil).
inline int stencil_prec32(const sgn_ctx* c) {
    return c->link_storage == SGN_LINKS_BF16 ? 2 : c->link_storage == SGN_LINKS_FP16 ? 3 : 1;
}
// Pick the fastest stencil launch shape for (precision, ncol) by timing candidates
// on the given buffers (ncol fields each); cached in the context.  Not during capture.
int tune_stencil(sgn_ctx* c, int prec, int ncol, void* in, void* out);
// Dot products <a_c, b_c> of ncol pairs of FP64 fields (host result, FP64 reductions).
int field_dots(sgn_ctx* c, const double2* a, const double2* b, int ncol, std::vector<std::complex<double>>& out);
// overlap operator D_ov = 1 + gamma5 F(A) (overlap.cu), packed fields
int overlap_apply(sgn_ctx* c, const double2* b, double2* y, int ncol, sgn_report* rep);
int overlap_solve(sgn_ctx* c, const double2* b, double2* x, int ncol, double tol, int k, int max_restarts,
                  int* iterations, double* relres);
// (A^2 - shift_col)^{-1} (I - Rp Lp^dag) rhs_col, one complex shift per column, restarted GMRES (FP64)
// x = x_P + ||r|| V_k sign(H_k) e_1 (eq. (6.3)) on packed FP64 fields; *kk_out = the
// largest Krylov dimension used (smaller than k only at a breakdown)
int direct_projection(sgn_ctx* c, const double2* b, double2* x, int ncol, int k, bool adjoint, int* kk_out);
int solve_columns_gmres(sgn_ctx* c, const double2* rhs, int ncol, const std::vector<std::complex<double>>& shift,
                        bool adjoint, double2* out, const double2* Rp, const double2* Lp, int mp);
int build_deflation(sgn_ctx* c, int m, int extra, double eig_tol, double* lambda_out);
// dH_W/dmu on ncol FP64 fields, and the mu-derivative of Re<g, x> (grad.cu).
cudaError_t apply_dhw_dmu64(const sgn_ctx* c, double2* out, const double2* in, int ncol, cudaStream_t st);
int grad_mu(sgn_ctx* c, const double2* b, const double2* g, int ncol, double* dmu);
void release_engines(sgn_ctx* c);

}  // namespace sgn
