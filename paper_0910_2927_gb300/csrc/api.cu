// The C ABI declared in include/sgn.h: argument checks, context state, host
// and device copies, stream ordering.  Numerical work lives in the kernels.
#include "ctx.cuh"

#include <cmath>
#include <cstring>
#include <new>

namespace sgn {

static thread_local std::string g_last_error;
thread_local long long g_launches = 0;

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

bool finite_host(const double* p, size_t count) {
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Order the internal stream after the caller's stream (entry) and the caller's
// stream after the internal one (exit).
int enter(sgn_ctx* c) {
    SGN_CUDA(cudaEventRecord(c->ev_in, c->user_stream));
    SGN_CUDA(cudaStreamWaitEvent(c->work, c->ev_in, 0));
    return SGN_OK;
}
int leave(sgn_ctx* c) {
    SGN_CUDA(cudaEventRecord(c->ev_out, c->work));
    SGN_CUDA(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
    return SGN_OK;
}

// One entry point's use of the work stream: close() orders the caller's stream after
// the work queued so far; an early error return does the same from the destructor, so
// the caller never runs ahead of kernels that still use its buffers.
struct Session {
    sgn_ctx* c;
    bool open = true;
    explicit Session(sgn_ctx* ctx) : c(ctx) {}
    ~Session() {
        if (open) leave(c);
    }
    int close() {
        open = false;
        return leave(c);
    }
};

// The operator changed: deflation data of the old operator no longer satisfy
// eq. (4.1).  They are dropped, and if there were any, the solves refuse to run
// until new data are set or built (or m = 0 is set explicitly).
int drop_deflation(sgn_ctx* c) {
    if (c->m > 0) c->deflation_stale = true;
    c->m = 0;
    c->lam.clear();
    c->mx = 0;
    c->lamx.clear();
    return SGN_OK;
}

// SGN_ERR_STATE while the deflation data belong to an operator that has since changed.
int check_deflation_current(const sgn_ctx* c, const char* who) {
    if (!c->deflation_stale) return SGN_OK;
    return fail(SGN_ERR_STATE, std::string(who) +
                                   ": the deflation data were dropped when the operator changed (gauge field, mu, "
                                   "kernel mass or boundary); build or set them again, or set m = 0");
}

int copy_in(sgn_ctx* c, void* dst, const void* src, size_t bytes, int on_device) {
    SGN_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->work));
    return SGN_OK;
}

// nfield natural-order complex128 fields (device, or host when on_device == 0)
// into packed device fields; host data pass through the staging buffer.
int fields_in(sgn_ctx* c, double2* packed, const double* src, int nfield, int on_device) {
    const double2* nat = reinterpret_cast<const double2*>(src);
    if (!on_device) {
        const size_t bytes = (size_t)c->n * nfield * sizeof(double2);
        SGN_CHECK(dev_alloc(c, c->stage, bytes));
        SGN_CUDA(cudaMemcpyAsync(c->stage.p, src, bytes, cudaMemcpyHostToDevice, c->work));
        nat = as<double2>(c->stage);
    }
    SGN_CUDA(pack_fields<double2>(nat, packed, c->vol, nfield, c->work));
    return SGN_OK;
}

}  // namespace
}  // namespace sgn

using namespace sgn;

SGN_API const char* sgn_last_error(void) { return g_last_error.c_str(); }

SGN_API const char* sgn_version(void) { return "sgn 0.1 (sm_103a)"; }

SGN_API int sgn_create(sgn_ctx** out, const int dims[4], sgn_alloc_fn alloc, sgn_free_fn free_, void* user,
                       void* stream) {
    if (!out || !dims) return fail(SGN_ERR_ARG, "sgn_create: NULL argument");
    *out = nullptr;
    for (int d = 0; d < 4; ++d)
        if (dims[d] < 2) return fail(SGN_ERR_ARG, "sgn_create: every lattice extent must be >= 2");
    if ((int64_t)dims[0] * dims[1] * dims[2] * dims[3] >= (int64_t(1) << 27))
        return fail(SGN_ERR_ARG, "sgn_create: the lattice volume must be below 2^27 sites");
    if ((alloc == nullptr) != (free_ == nullptr))
        return fail(SGN_ERR_ARG, "sgn_create: give both allocator callbacks or neither");
    sgn_ctx* c = new (std::nothrow) sgn_ctx();
    if (!c) return fail(SGN_ERR_ALLOC, "sgn_create: out of host memory");
    for (int d = 0; d < 4; ++d) c->dims[d] = dims[d];
    c->vol = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    c->n = 12 * c->vol;
    c->alloc = alloc;
    c->free_ = free_;
    c->user = user;
    c->user_stream = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_t1);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_k0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev_k1);
    if (e == cudaSuccess) e = prepare_small_kernels();
    if (e != cudaSuccess) {
        set_error(std::string("sgn_create: ") + cudaGetErrorString(e));
        sgn_destroy(c);
        return SGN_ERR_CUDA;
    }
    *out = c;
    return SGN_OK;
}

SGN_API int sgn_destroy(sgn_ctx* c) {
    if (!c) return SGN_OK;
    if (c->work) cudaStreamSynchronize(c->work);
    release_engines(c);
    dev_free(c, c->U64);
    dev_free(c, c->U32);
    dev_free(c, c->U16);
    dev_free(c, c->UH);
    dev_free(c, c->Uff);
    dev_free(c, c->R64);
    dev_free(c, c->L64);
    dev_free(c, c->R32);
    dev_free(c, c->L32);
    dev_free(c, c->lam_dev);
    dev_free(c, c->lamc_dev);
    dev_free(c, c->Rx64);
    dev_free(c, c->Lx64);
    dev_free(c, c->io);
    dev_free(c, c->stage);
    dev_free(c, c->ip_scratch);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ev_t0) cudaEventDestroy(c->ev_t0);
    if (c->ev_t1) cudaEventDestroy(c->ev_t1);
    if (c->ev_k0) cudaEventDestroy(c->ev_k0);
    if (c->ev_k1) cudaEventDestroy(c->ev_k1);
    if (c->work) cudaStreamDestroy(c->work);
    delete c;
    return SGN_OK;
}

SGN_API int sgn_set_stream(sgn_ctx* c, void* stream) {
    if (!c) return fail(SGN_ERR_ARG, "sgn_set_stream: NULL context");
    c->user_stream = reinterpret_cast<cudaStream_t>(stream);
    return SGN_OK;
}

SGN_API int sgn_load_gauge(sgn_ctx* c, const double* links, int on_device) {
    if (!c || !links) return fail(SGN_ERR_ARG, "sgn_load_gauge: NULL argument");
    const size_t count = (size_t)c->vol * 36;  // complex entries
    if (!on_device && !finite_host(links, 2 * count))
        return fail(SGN_ERR_NONFINITE, "sgn_load_gauge: non-finite link entry");
    SGN_CHECK(enter(c));
    Session ses(c);
    SGN_CHECK(dev_alloc(c, c->U64, count * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->U32, count * sizeof(float2)));
    SGN_CHECK(dev_alloc(c, c->U16, count * sizeof(__nv_bfloat162)));
    SGN_CHECK(dev_alloc(c, c->UH, count * sizeof(__half2)));
    SGN_CHECK(dev_alloc(c, c->Uff, count * sizeof(float4)));
    const double2* nat = reinterpret_cast<const double2*>(links);
    if (!on_device) {
        SGN_CHECK(dev_alloc(c, c->stage, count * sizeof(double2)));
        SGN_CHECK(copy_in(c, c->stage.p, links, count * sizeof(double2), 0));
        nat = as<double2>(c->stage);
    }
    SGN_CUDA(pack_links(nat, as<double2>(c->U64), c->vol, c->work));
    SGN_CUDA(convert_f64_to_f32(as<double2>(c->U64), as<float2>(c->U32), (int64_t)count, c->work));
    SGN_CUDA(links_f64_to_bf16(as<double2>(c->U64), as<__nv_bfloat162>(c->U16), (int64_t)count, c->work));
    SGN_CUDA(links_f64_to_f16(as<double2>(c->U64), as<__half2>(c->UH), (int64_t)count, c->work));
    SGN_CUDA(links_ff(as<double2>(c->U64), as<float2>(c->U32), as<float4>(c->Uff), (int64_t)count, c->work));
    SGN_CUDA(cudaStreamSynchronize(c->work));
    SGN_CHECK(ses.close());
    c->have_gauge = true;
    drop_deflation(c);
    return SGN_OK;
}

SGN_API int sgn_set_mu(sgn_ctx* c, double mu) {
    if (!c || !std::isfinite(mu)) return fail(SGN_ERR_ARG, "sgn_set_mu: bad argument");
    if (mu != c->mu) drop_deflation(c);
    c->mu = mu;
    return SGN_OK;
}

SGN_API int sgn_set_kernel_mass(sgn_ctx* c, double m_w) {
    if (!c || !std::isfinite(m_w)) return fail(SGN_ERR_ARG, "sgn_set_kernel_mass: bad argument");
    if (m_w != c->mass) drop_deflation(c);
    c->mass = m_w;
    return SGN_OK;
}

SGN_API int sgn_set_boundary(sgn_ctx* c, const int antiperiodic[4]) {
    if (!c || !antiperiodic) return fail(SGN_ERR_ARG, "sgn_set_boundary: NULL argument");
    bool changed = false;
    for (int d = 0; d < 4; ++d) {
        int v = antiperiodic[d] ? 1 : 0;
        changed = changed || v != c->ap[d];
        c->ap[d] = v;
    }
    if (changed) drop_deflation(c);
    return SGN_OK;
}

SGN_API int sgn_kenney_laub(int s, double c, double* sigma, double* omega) {
    if (s < 1 || !(c > 0) || !std::isfinite(c) || !sigma || !omega)
        return fail(SGN_ERR_ARG, "sgn_kenney_laub: need s >= 1, finite c > 0 and output arrays");
    // eq. (6.2): theta_i = (pi / 2s)(i - 1/2), i = 1..s
    for (int i = 0; i < s; ++i) {
        const double th = M_PI * (i + 0.5) / (2.0 * s);
        const double t = std::tan(th), co = std::cos(th);
        sigma[i] = -(t * t) / (c * c);
        omega[i] = 1.0 / (s * co * co * c);
    }
    return SGN_OK;
}

SGN_API int sgn_set_rational(sgn_ctx* c, int s, const double* sigma, const double* omega) {
    if (!c || !sigma || !omega || s < 1 || s > 32) return fail(SGN_ERR_ARG, "sgn_set_rational: need 1 <= s <= 32");
    if (!finite_host(sigma, s) || !finite_host(omega, s))
        return fail(SGN_ERR_ARG, "sgn_set_rational: non-finite shift or weight");
    c->sigma.assign(sigma, sigma + s);
    c->omega.assign(omega, omega + s);
    return SGN_OK;
}

SGN_API int sgn_set_restart(sgn_ctx* c, int k, double tol, int max_cycles, int project_each_cycle) {
    if (!c || k < 1 || k > 64 || !(tol > 0) || max_cycles < 1)
        return fail(SGN_ERR_ARG, "sgn_set_restart: need 1 <= k <= 64, tol > 0, max_cycles >= 1");
    c->k = k;
    c->tol = tol;
    c->max_cycles = max_cycles;
    c->project = project_each_cycle ? 1 : 0;
    return SGN_OK;
}

SGN_API int sgn_set_precision(sgn_ctx* c, int precision, double target_rel_err, int link_storage) {
    if (!c || (precision != SGN_PREC_FP64 && precision != SGN_PREC_MIXED) || !(target_rel_err > 0) ||
        (link_storage != SGN_LINKS_FP32 && link_storage != SGN_LINKS_BF16 && link_storage != SGN_LINKS_FP16))
        return fail(SGN_ERR_ARG, "sgn_set_precision: bad argument");
    c->precision = precision;
    c->target = target_rel_err;
    c->link_storage = link_storage;
    return SGN_OK;
}

SGN_API int sgn_set_formulation(sgn_ctx* c, int form) {
    if (!c || (form != SGN_FORM_A2 && form != SGN_FORM_A)) return fail(SGN_ERR_ARG, "sgn_set_formulation: bad argument");
    c->form = form;
    return SGN_OK;
}

SGN_API int sgn_set_method(sgn_ctx* c, int method) {
    if (!c || (method != SGN_METHOD_FOM && method != SGN_METHOD_GMRES))
        return fail(SGN_ERR_ARG, "sgn_set_method: bad argument");
    c->method = method;
    return SGN_OK;
}

SGN_API int sgn_set_refinement(sgn_ctx* c, int k_refine, int max_batch) {
    if (!c || k_refine < 0 || k_refine > 64 || max_batch < 0 || max_batch > 4096)
        return fail(SGN_ERR_ARG, "sgn_set_refinement: need 0 <= k_refine <= 64, 0 <= max_batch <= 4096");
    c->k_refine = k_refine;
    c->refine_batch = max_batch;
    return SGN_OK;
}

SGN_API int sgn_set_deflation(sgn_ctx* c, int m, const double* R, const double* L, const double* lambda,
                              int on_device) {
    if (!c || m < 0 || m > 64) return fail(SGN_ERR_ARG, "sgn_set_deflation: need 0 <= m <= 64");
    if (m == 0) {
        drop_deflation(c);
        c->deflation_stale = false;  // an explicit choice of no deflation
        return SGN_OK;
    }
    if (!R || !L || !lambda) return fail(SGN_ERR_ARG, "sgn_set_deflation: NULL argument");
    const size_t cnt = (size_t)c->n * m;
    std::vector<double> lam(2 * (size_t)m);
    if (on_device) {
        SGN_CUDA(cudaMemcpy(lam.data(), lambda, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(lam.data(), lambda, sizeof(double) * 2 * m);
        if (!finite_host(R, 2 * cnt) || !finite_host(L, 2 * cnt))
            return fail(SGN_ERR_NONFINITE, "sgn_set_deflation: non-finite vector entry");
    }
    if (!finite_host(lam.data(), 2 * (size_t)m)) return fail(SGN_ERR_NONFINITE, "sgn_set_deflation: bad lambda");
    for (int j = 0; j < m; ++j)
        if (lam[2 * j] == 0.0)
            return fail(SGN_ERR_DEFLATION, "sgn_set_deflation: an eigenvalue on the imaginary axis has no sign");
    SGN_CHECK(enter(c));
    Session ses(c);
    SGN_CHECK(dev_alloc(c, c->R64, cnt * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->L64, cnt * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->R32, cnt * sizeof(float2)));
    SGN_CHECK(dev_alloc(c, c->L32, cnt * sizeof(float2)));
    SGN_CHECK(dev_alloc(c, c->lam_dev, (size_t)m * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->lamc_dev, (size_t)m * sizeof(double2)));
    SGN_CHECK(fields_in(c, as<double2>(c->R64), R, m, on_device));
    SGN_CHECK(fields_in(c, as<double2>(c->L64), L, m, on_device));
    SGN_CUDA(convert_f64_to_f32(as<double2>(c->R64), as<float2>(c->R32), (int64_t)cnt, c->work));
    SGN_CUDA(convert_f64_to_f32(as<double2>(c->L64), as<float2>(c->L32), (int64_t)cnt, c->work));
    std::vector<double> lamc(lam);
    for (int j = 0; j < m; ++j) lamc[2 * j + 1] = -lamc[2 * j + 1];
    SGN_CUDA(cudaMemcpyAsync(c->lam_dev.p, lam.data(), sizeof(double) * 2 * m, cudaMemcpyHostToDevice, c->work));
    SGN_CUDA(cudaMemcpyAsync(c->lamc_dev.p, lamc.data(), sizeof(double) * 2 * m, cudaMemcpyHostToDevice, c->work));
    SGN_CUDA(cudaStreamSynchronize(c->work));
    SGN_CHECK(ses.close());
    c->lam.resize(m);
    for (int j = 0; j < m; ++j) c->lam[j] = {lam[2 * j], lam[2 * j + 1]};
    c->m = m;
    c->deflation_stale = false;
    return SGN_OK;
}

SGN_API int sgn_set_deflation_extra(sgn_ctx* c, int e, const double* R, const double* L, const double* lambda,
                                    int on_device) {
    if (!c || e < 0 || e > 64) return fail(SGN_ERR_ARG, "sgn_set_deflation_extra: need 0 <= e <= 64");
    if (e == 0) {
        c->mx = 0;
        c->lamx.clear();
        return SGN_OK;
    }
    if (!R || !L || !lambda) return fail(SGN_ERR_ARG, "sgn_set_deflation_extra: NULL argument");
    const size_t cnt = (size_t)c->n * e;
    std::vector<double> lam(2 * (size_t)e);
    if (on_device) {
        SGN_CUDA(cudaMemcpy(lam.data(), lambda, sizeof(double) * 2 * e, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(lam.data(), lambda, sizeof(double) * 2 * e);
        if (!finite_host(R, 2 * cnt) || !finite_host(L, 2 * cnt))
            return fail(SGN_ERR_NONFINITE, "sgn_set_deflation_extra: non-finite vector entry");
    }
    if (!finite_host(lam.data(), 2 * (size_t)e)) return fail(SGN_ERR_NONFINITE, "sgn_set_deflation_extra: bad lambda");
    SGN_CHECK(enter(c));
    Session ses(c);
    SGN_CHECK(dev_alloc(c, c->Rx64, cnt * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->Lx64, cnt * sizeof(double2)));
    SGN_CHECK(fields_in(c, as<double2>(c->Rx64), R, e, on_device));
    SGN_CHECK(fields_in(c, as<double2>(c->Lx64), L, e, on_device));
    SGN_CUDA(cudaStreamSynchronize(c->work));
    SGN_CHECK(ses.close());
    c->lamx.resize(e);
    for (int j = 0; j < e; ++j) c->lamx[j] = {lam[2 * j], lam[2 * j + 1]};
    c->mx = e;
    return SGN_OK;
}

SGN_API int sgn_get_deflation(sgn_ctx* c, int* m, double* R, double* L, double* lambda) {
    if (!c) return fail(SGN_ERR_ARG, "sgn_get_deflation: NULL context");
    if (m) *m = c->m;
    if (c->m == 0) return SGN_OK;
    const size_t cnt = (size_t)c->n * c->m;
    SGN_CHECK(enter(c));
    Session ses(c);
    SGN_CHECK(dev_alloc(c, c->stage, cnt * sizeof(double2)));
    for (int side = 0; side < 2; ++side) {
        double* dst = side == 0 ? R : L;
        if (!dst) continue;
        SGN_CUDA(unpack_fields<double2>(as<double2>(side == 0 ? c->R64 : c->L64), as<double2>(c->stage), c->vol,
                                        c->m, c->work));
        SGN_CUDA(cudaMemcpyAsync(dst, c->stage.p, cnt * sizeof(double2), cudaMemcpyDeviceToHost, c->work));
        SGN_CUDA(cudaStreamSynchronize(c->work));
    }
    SGN_CHECK(ses.close());
    if (lambda)
        for (int j = 0; j < c->m; ++j) {
            lambda[2 * j] = c->lam[j].real();
            lambda[2 * j + 1] = c->lam[j].imag();
        }
    return SGN_OK;
}

SGN_API int sgn_build_deflation(sgn_ctx* c, int m, int extra, double eig_tol, double* lambda_out) {
    if (!c || m < 1 || m > 64 || extra < 0 || m + extra > 64 || !(eig_tol > 0))
        return fail(SGN_ERR_ARG, "sgn_build_deflation: need 1 <= m, m + extra <= 64, eig_tol > 0");
    if (!c->have_gauge) return fail(SGN_ERR_STATE, "sgn_build_deflation: load the gauge field first");
    SGN_CHECK(enter(c));
    Session ses(c);
    int st = build_deflation(c, m, extra, eig_tol, lambda_out);
    SGN_CHECK(ses.close());
    return st;
}

namespace {

int apply_common(sgn_ctx* c, const double* b, double* x, double* x_shift, int nrhs, int flags, sgn_report* rep) {
    if (!c || !b || !x || nrhs < 1) return fail(SGN_ERR_ARG, "sgn_apply: bad argument");
    if (!c->have_gauge) return fail(SGN_ERR_STATE, "sgn_apply: load the gauge field first");
    if (c->sigma.empty()) return fail(SGN_ERR_STATE, "sgn_apply: set the rational function first");
    SGN_CHECK(check_deflation_current(c, "sgn_apply"));
    if (x_shift && (flags & SGN_APPLY_HOST_BUFFERS))
        return fail(SGN_ERR_ARG, "sgn_apply_shifts: per-shift output needs device buffers");
    const bool host = flags & SGN_APPLY_HOST_BUFFERS;
    const bool adjoint = flags & SGN_APPLY_ADJOINT;
    const size_t fbytes = (size_t)c->n * nrhs * sizeof(double2);
    if (host && !finite_host(b, 2 * (size_t)c->n * nrhs))
        return fail(SGN_ERR_NONFINITE, "sgn_apply: non-finite entry in b");
    SGN_CHECK(enter(c));
    Session ses(c);
    const long long launches0 = g_launches;
    SGN_CUDA(cudaEventRecord(c->ev_t0, c->work));
    // staging: [b packed][x packed][x_shift packed]
    const size_t nn = (size_t)c->n * nrhs;
    const int s = (int)c->sigma.size();
    SGN_CHECK(dev_alloc(c, c->stage, (2 + (x_shift ? s : 0)) * fbytes));
    double2* bp = as<double2>(c->stage);
    double2* xp = bp + nn;
    double2* xsp = x_shift ? xp + nn : nullptr;
    if (host) {  // natural b lands in the x slot, is packed into the b slot
        SGN_CUDA(cudaMemcpyAsync(xp, b, fbytes, cudaMemcpyHostToDevice, c->work));
        SGN_CUDA(pack_fields<double2>(xp, bp, c->vol, nrhs, c->work));
    } else {
        SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(b), bp, c->vol, nrhs, c->work));
    }
    const bool no_a = flags & SGN_APPLY_NO_A;
    int status = solve(c, bp, xp, xsp, nrhs, adjoint, no_a, rep);
    if (status == SGN_OK || status == SGN_ERR_NOT_CONVERGED) {
        if (host) {  // natural x goes out through the b slot
            SGN_CUDA(unpack_fields<double2>(xp, bp, c->vol, nrhs, c->work));
            SGN_CUDA(cudaMemcpyAsync(x, bp, fbytes, cudaMemcpyDeviceToHost, c->work));
        } else {
            SGN_CUDA(unpack_fields<double2>(xp, reinterpret_cast<double2*>(x), c->vol, nrhs, c->work));
            if (xsp)
                SGN_CUDA(unpack_fields<double2>(xsp, reinterpret_cast<double2*>(x_shift), c->vol, s * nrhs,
                                                c->work));
        }
    }
    SGN_CUDA(cudaEventRecord(c->ev_t1, c->work));
    SGN_CUDA(cudaEventSynchronize(c->ev_t1));
    if (rep) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev_t0, c->ev_t1);
        rep->ms = ms;
        rep->kernels = g_launches - launches0;
    }
    SGN_CHECK(ses.close());
    return status;
}

}  // namespace

SGN_API int sgn_apply(sgn_ctx* c, const double* b, double* x, int nrhs, int flags, sgn_report* rep) {
    return apply_common(c, b, x, nullptr, nrhs, flags, rep);
}

SGN_API int sgn_apply_shifts(sgn_ctx* c, const double* b, double* x, double* x_shift, int nrhs, int flags,
                             sgn_report* rep) {
    if (!x_shift) return fail(SGN_ERR_ARG, "sgn_apply_shifts: NULL x_shift");
    return apply_common(c, b, x, x_shift, nrhs, flags, rep);
}

SGN_API int sgn_hw_apply(sgn_ctx* c, const void* in, void* out, int nrhs, int precision, int flags) {
    if (!c || !in || !out || nrhs < 1) return fail(SGN_ERR_ARG, "sgn_hw_apply: bad argument");
    if (in == out) return fail(SGN_ERR_ARG, "sgn_hw_apply: in and out must differ");
    if (!c->have_gauge) return fail(SGN_ERR_STATE, "sgn_hw_apply: load the gauge field first");
    if (precision != SGN_PREC_FP64 && precision != SGN_PREC_MIXED)
        return fail(SGN_ERR_ARG, "sgn_hw_apply: unknown precision");
    if (flags & ~(SGN_HW_ADJOINT | SGN_HW_PACKED | SGN_HW_FLOAT_FLOAT))
        return fail(SGN_ERR_ARG, "sgn_hw_apply: unknown flag");
    const bool adjoint = flags & SGN_HW_ADJOINT;
    const bool packed = flags & SGN_HW_PACKED;
    const bool ffa = flags & SGN_HW_FLOAT_FLOAT;
    if (ffa && precision != SGN_PREC_FP64)
        return fail(SGN_ERR_ARG, "sgn_hw_apply: SGN_HW_FLOAT_FLOAT takes complex128 fields (SGN_PREC_FP64)");
    SGN_CHECK(enter(c));
    Session ses(c);
    const size_t nn = (size_t)c->n * nrhs;
    if (precision == SGN_PREC_FP64) {
        const double2* pi = reinterpret_cast<const double2*>(in);
        double2* po = reinterpret_cast<double2*>(out);
        // staging (complex128 units): the packed copies of in and out, then the float-float
        // (hi, lo) pairs of in and out (4 nn complex64 = 2 nn complex128)
        const size_t need = (packed ? 0 : 2 * nn) + (ffa ? 2 * nn : 0);
        double2* t = nullptr;
        if (need) {
            SGN_CHECK(dev_alloc(c, c->stage, need * sizeof(double2)));
            t = as<double2>(c->stage);
        }
        if (!packed) {
            SGN_CUDA(pack_fields<double2>(pi, t, c->vol, nrhs, c->work));
            pi = t;
            po = t + nn;
        }
        if (ffa) {
            float2* f = reinterpret_cast<float2*>(t + (packed ? 0 : 2 * nn));
            float2 *ih = f, *il = f + nn, *oh = f + 2 * nn, *ol = f + 3 * nn;
            SGN_CUDA(split_ff(pi, ih, il, (int64_t)nn, c->work));
            SGN_CUDA(launch_hw_ff(oh, ol, ih, il, as<float4>(c->Uff), nrhs, stencil_params(c, adjoint), c->work));
            SGN_CUDA(join_ff(oh, ol, po, (int64_t)nn, c->work));
        } else {
            SGN_CHECK(tune_stencil(c, 0, nrhs, const_cast<double2*>(pi), po));
            SGN_CUDA(apply_hw64(c, po, pi, nrhs, adjoint, nullptr, c->work));
        }
        if (!packed)
            SGN_CUDA(unpack_fields<double2>(po, reinterpret_cast<double2*>(out), c->vol, nrhs, c->work));
    } else {
        const float2* pi = reinterpret_cast<const float2*>(in);
        float2* po = reinterpret_cast<float2*>(out);
        if (!packed) {
            SGN_CHECK(dev_alloc(c, c->stage, 2 * nn * sizeof(float2)));
            float2* t = as<float2>(c->stage);
            SGN_CUDA(pack_fields<float2>(pi, t, c->vol, nrhs, c->work));
            pi = t;
            po = t + nn;
        }
        SGN_CHECK(tune_stencil(c, stencil_prec32(c), nrhs, const_cast<float2*>(pi), po));
        SGN_CUDA(apply_hw32(c, po, pi, nrhs, adjoint, nullptr, c->work));
        if (!packed)
            SGN_CUDA(unpack_fields<float2>(po, reinterpret_cast<float2*>(out), c->vol, nrhs, c->work));
    }
    SGN_CHECK(ses.close());
    return SGN_OK;
}

SGN_API int sgn_overlap_apply(sgn_ctx* c, const double* b, double* y, int nrhs) {
    if (!c || !b || !y || nrhs < 1 || b == y) return fail(SGN_ERR_ARG, "sgn_overlap_apply: bad argument");
    if (!c->have_gauge || c->sigma.empty()) return fail(SGN_ERR_STATE, "sgn_overlap_apply: gauge field and rational function needed");
    SGN_CHECK(check_deflation_current(c, "sgn_overlap_apply"));
    SGN_CHECK(enter(c));
    Session ses(c);
    const size_t nn = (size_t)c->n * nrhs;
    SGN_CHECK(dev_alloc(c, c->stage, 2 * nn * sizeof(double2)));
    double2* t = as<double2>(c->stage);
    SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(b), t, c->vol, nrhs, c->work));
    int st = overlap_apply(c, t, t + nn, nrhs, nullptr);
    if (st == SGN_OK) SGN_CUDA(unpack_fields<double2>(t + nn, reinterpret_cast<double2*>(y), c->vol, nrhs, c->work));
    SGN_CHECK(ses.close());
    return st;
}

SGN_API int sgn_overlap_solve(sgn_ctx* c, const double* b, double* x, int nrhs, double tol, int k, int max_restarts,
                              int* iterations, double* relres) {
    if (!c || !b || !x || nrhs < 1 || b == x || !(tol > 0) || k < 1 || k > 64 || max_restarts < 0)
        return fail(SGN_ERR_ARG, "sgn_overlap_solve: need tol > 0, 1 <= k <= 64, max_restarts >= 0");
    if (!c->have_gauge || c->sigma.empty()) return fail(SGN_ERR_STATE, "sgn_overlap_solve: gauge field and rational function needed");
    SGN_CHECK(check_deflation_current(c, "sgn_overlap_solve"));
    SGN_CHECK(enter(c));
    Session ses(c);
    const size_t nn = (size_t)c->n * nrhs;
    SGN_CHECK(dev_alloc(c, c->stage, 2 * nn * sizeof(double2)));
    double2* t = as<double2>(c->stage);
    SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(b), t, c->vol, nrhs, c->work));
    SGN_CUDA(cudaMemsetAsync(t + nn, 0, nn * sizeof(double2), c->work));  // initial guess 0
    int st = overlap_solve(c, t, t + nn, nrhs, tol, k, max_restarts, iterations, relres);
    if (st == SGN_OK || st == SGN_ERR_NOT_CONVERGED)
        SGN_CUDA(unpack_fields<double2>(t + nn, reinterpret_cast<double2*>(x), c->vol, nrhs, c->work));
    SGN_CHECK(ses.close());
    return st;
}

SGN_API int sgn_apply_direct(sgn_ctx* c, const double* b, double* x, int nrhs, int k, int flags, int* k_used) {
    if (!c || !b || !x || nrhs < 1 || b == x || k < 1 || k > 4096)
        return fail(SGN_ERR_ARG, "sgn_apply_direct: need b != x, nrhs >= 1, 1 <= k <= 4096");
    if (flags & ~SGN_APPLY_ADJOINT) return fail(SGN_ERR_ARG, "sgn_apply_direct: unknown flag");
    if (!c->have_gauge) return fail(SGN_ERR_STATE, "sgn_apply_direct: load the gauge field first");
    SGN_CHECK(check_deflation_current(c, "sgn_apply_direct"));
    SGN_CHECK(enter(c));
    Session ses(c);
    const size_t nn = (size_t)c->n * nrhs;
    SGN_CHECK(dev_alloc(c, c->stage, 2 * nn * sizeof(double2)));
    double2* t = as<double2>(c->stage);
    SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(b), t, c->vol, nrhs, c->work));
    SGN_CHECK(tune_stencil(c, 0, nrhs, t, t + nn));
    int st = direct_projection(c, t, t + nn, nrhs, k, (flags & SGN_APPLY_ADJOINT) != 0, k_used);
    if (st == SGN_OK) SGN_CUDA(unpack_fields<double2>(t + nn, reinterpret_cast<double2*>(x), c->vol, nrhs, c->work));
    SGN_CHECK(ses.close());
    return st;
}

SGN_API int sgn_pack_fields(sgn_ctx* c, const void* in, void* out, int nfield, int precision) {
    if (!c || !in || !out || nfield < 1 || nfield > 65535) return fail(SGN_ERR_ARG, "sgn_pack_fields: bad argument");
    if (in == out) return fail(SGN_ERR_ARG, "sgn_pack_fields: in and out must differ");
    if (precision != SGN_PREC_FP64 && precision != SGN_PREC_MIXED)
        return fail(SGN_ERR_ARG, "sgn_pack_fields: unknown precision");
    SGN_CHECK(enter(c));
    Session ses(c);
    if (precision == SGN_PREC_FP64)
        SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out), c->vol,
                                      nfield, c->work));
    else
        SGN_CUDA(pack_fields<float2>(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), c->vol,
                                     nfield, c->work));
    SGN_CHECK(ses.close());
    return SGN_OK;
}

SGN_API int sgn_unpack_fields(sgn_ctx* c, const void* in, void* out, int nfield, int precision) {
    if (!c || !in || !out || nfield < 1 || nfield > 65535)
        return fail(SGN_ERR_ARG, "sgn_unpack_fields: bad argument");
    if (in == out) return fail(SGN_ERR_ARG, "sgn_unpack_fields: in and out must differ");
    if (precision != SGN_PREC_FP64 && precision != SGN_PREC_MIXED)
        return fail(SGN_ERR_ARG, "sgn_unpack_fields: unknown precision");
    SGN_CHECK(enter(c));
    Session ses(c);
    if (precision == SGN_PREC_FP64)
        SGN_CUDA(unpack_fields<double2>(reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out),
                                        c->vol, nfield, c->work));
    else
        SGN_CUDA(unpack_fields<float2>(reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), c->vol,
                                       nfield, c->work));
    SGN_CHECK(ses.close());
    return SGN_OK;
}

SGN_API int sgn_dhw_dmu_apply(sgn_ctx* c, const double* in, double* out, int nrhs) {
    if (!c || !in || !out || nrhs < 1) return fail(SGN_ERR_ARG, "sgn_dhw_dmu_apply: bad argument");
    if (in == out) return fail(SGN_ERR_ARG, "sgn_dhw_dmu_apply: in and out must differ");
    if (!c->have_gauge) return fail(SGN_ERR_STATE, "sgn_dhw_dmu_apply: load the gauge field first");
    SGN_CHECK(enter(c));
    Session ses(c);
    const size_t nn = (size_t)c->n * nrhs;
    SGN_CHECK(dev_alloc(c, c->stage, 2 * nn * sizeof(double2)));
    double2* t = as<double2>(c->stage);
    SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(in), t, c->vol, nrhs, c->work));
    SGN_CUDA(apply_dhw_dmu64(c, t + nn, t, nrhs, c->work));
    SGN_CUDA(unpack_fields<double2>(t + nn, reinterpret_cast<double2*>(out), c->vol, nrhs, c->work));
    SGN_CHECK(ses.close());
    return SGN_OK;
}

SGN_API int sgn_grad_mu(sgn_ctx* c, const double* b, const double* g, int nrhs, double* dmu) {
    if (!c || !b || !g || !dmu || nrhs < 1) return fail(SGN_ERR_ARG, "sgn_grad_mu: bad argument");
    if (!c->have_gauge || c->sigma.empty()) return fail(SGN_ERR_STATE, "sgn_grad_mu: gauge field and rational function needed");
    if (c->form != SGN_FORM_A2) return fail(SGN_ERR_STATE, "sgn_grad_mu: needs the A^2 formulation (per-shift iterates)");
    SGN_CHECK(check_deflation_current(c, "sgn_grad_mu"));
    SGN_CHECK(enter(c));
    Session ses(c);
    const size_t nn = (size_t)c->n * nrhs;
    SGN_CHECK(dev_alloc(c, c->stage, 2 * nn * sizeof(double2)));
    double2* t = as<double2>(c->stage);
    SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(b), t, c->vol, nrhs, c->work));
    SGN_CUDA(pack_fields<double2>(reinterpret_cast<const double2*>(g), t + nn, c->vol, nrhs, c->work));
    int st = grad_mu(c, t, t + nn, nrhs, dmu);
    SGN_CHECK(ses.close());
    return st;
}

SGN_API int sgn_inner_products(sgn_ctx* c, const double* V, int J, const double* w, int nrhs, double* out) {
    if (!c || !V || !w || !out || J < 1 || J > 64 || nrhs < 1)
        return fail(SGN_ERR_ARG, "sgn_inner_products: need 1 <= J <= 64, nrhs >= 1 and non-NULL pointers");
    SGN_CHECK(enter(c));
    Session ses(c);
    const int64_t n = c->n;
    const int nblk = reduce_blocks<double2>(n);
    const int rs = (J + 8) & ~7;
    const size_t pbytes = (sizeof(double2) * (size_t)nrhs * rs * nblk + 255) & ~size_t(255);
    const size_t rbytes = (sizeof(double2) * (size_t)nrhs * rs + 255) & ~size_t(255);
    SGN_CHECK(dev_alloc(c, c->ip_scratch, pbytes + rbytes + sizeof(int) * 2 * nrhs));
    char* p = reinterpret_cast<char*>(c->ip_scratch.p);
    DevState S{};
    S.red = reinterpret_cast<double2*>(p + pbytes);
    S.skip = reinterpret_cast<int*>(p + pbytes + rbytes);
    S.done = S.skip + nrhs;
    S.rstride = rs;
    SGN_CUDA(cudaMemsetAsync(S.skip, 0, sizeof(int) * 2 * nrhs, c->work));
    const Reduce rd{reinterpret_cast<double2*>(p), nblk, rs};
    SGN_CUDA(mdot<double2>(Basis<double2>{reinterpret_cast<const double2*>(V), n, 0}, J,
                           reinterpret_cast<const double2*>(w), n, n, nrhs, rd, 0, nullptr, c->work));
    SGN_CUDA(reduce(rd, J, nrhs, RM_STORE, 0, S, nullptr, c->work));
    std::vector<double2> h((size_t)nrhs * rs);
    SGN_CUDA(cudaMemcpyAsync(h.data(), S.red, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, c->work));
    SGN_CUDA(cudaStreamSynchronize(c->work));
    SGN_CHECK(ses.close());
    for (int col = 0; col < nrhs; ++col)
        for (int j = 0; j < J; ++j) {
            out[2 * ((size_t)col * J + j)] = h[(size_t)col * rs + j].x;
            out[2 * ((size_t)col * J + j) + 1] = h[(size_t)col * rs + j].y;
        }
    return SGN_OK;
}

SGN_API int sgn_get_hessenberg(sgn_ctx* c, int col, double* H, int* k_used) {
    if (!c || col < 0) return fail(SGN_ERR_ARG, "sgn_get_hessenberg: bad argument");
    Engine* E = c->last_fp64;
    if (!E) return fail(SGN_ERR_STATE, "sgn_get_hessenberg: no FP64-form solve has run");
    if (col >= E->ncol) return fail(SGN_ERR_ARG, "sgn_get_hessenberg: column out of range");
    const int km = E->S.kmax;
    SGN_CHECK(enter(c));
    Session ses(c);
    int kk = 0;
    SGN_CUDA(cudaMemcpyAsync(&kk, E->S.kk + col, sizeof(int), cudaMemcpyDeviceToHost, c->work));
    if (H)
        SGN_CUDA(cudaMemcpyAsync(H, E->S.H + (size_t)col * (km + 1) * km, sizeof(double2) * (size_t)(km + 1) * km,
                                 cudaMemcpyDeviceToHost, c->work));
    SGN_CUDA(cudaStreamSynchronize(c->work));
    SGN_CHECK(ses.close());
    if (k_used) *k_used = kk;
    return SGN_OK;
}

SGN_API int sgn_set_kernel_timing(sgn_ctx* c, int on) {
    if (!c) return fail(SGN_ERR_ARG, "sgn_set_kernel_timing: NULL context");
    c->timing = on ? 1 : 0;
    for (int i = 0; i < sgn_ctx::kTimedClasses; ++i) {
        c->t_ms[i] = 0;
        c->t_launches[i] = 0;
        c->t_bytes[i] = 0;
    }
    return SGN_OK;
}

SGN_API int sgn_get_kernel_timing(sgn_ctx* c, int cls, double* ms, long long* launches, double* bytes) {
    if (!c || cls < 0 || cls >= sgn_ctx::kTimedClasses) return fail(SGN_ERR_ARG, "sgn_get_kernel_timing: bad argument");
    if (ms) *ms = c->t_ms[cls];
    if (launches) *launches = c->t_launches[cls];
    if (bytes) *bytes = c->t_bytes[cls];
    return SGN_OK;
}
