/*
 * sgn.h -- C ABI of the GB300 library for sign(H_W(mu)) b.
 *
 * Method: Bloch, Breu, Frommer, Heybrock, Schaefer, Wettig, "Krylov subspace
 * methods and the sign function: multishifts and deflation in the
 * non-Hermitian case" (Lattice 2009).  The library computes
 *
 *     x = R sign(Re Lambda) L^dag b + sum_i omega_i (A^2 - sigma_i)^{-1} A (I - P) b
 *
 * for A = H_W(mu) = gamma5 D_W(mu) (Sec. 1), P = R L^dag (Sec. 4, eqs. (4.1)-(4.3)),
 * and the partial fractions of eq. (6.2), by restarted LR-deflated multishift
 * FOM (Algorithm 1, "FOM-LR(m,k)") run on A^2 with right-hand side A (I - P) b.
 *
 * Conventions shared by every call
 * --------------------------------
 *  * Lattice dims = {Lx, Ly, Lz, Lt}; site = x + Lx*(y + Ly*(z + Lz*t)); V = Lx*Ly*Lz*Lt.
 *  * Spinor field: V*12 complex numbers, [site][spin 4][colour 3], complex stored
 *    as interleaved (re, im) pairs.  "nrhs fields" are nrhs such fields back to back.
 *  * Gauge links: V*4*9 complex128, [site][dir x,y,z,t][row 3][col 3].
 *  * D_W(mu) psi(x) = (4 + m_W) psi(x) - 1/2 sum_nu [(1 - gamma_nu) e^{+mu d_nu,t} U_nu(x) psi(x+nu)
 *                    + (1 + gamma_nu) e^{-mu d_nu,t} U_nu(x-nu)^dag psi(x-nu)],
 *    chiral Euclidean gamma matrices, gamma5 = diag(1, 1, -1, -1) in spin.
 *  * Every call returns an sgn_status (0 = success); no C++ exception crosses
 *    the ABI.  On failure sgn_last_error() returns a thread-local message.
 *  * All device work runs on the stream given to sgn_create (or sgn_set_stream).
 *    Calls that return results to the host synchronise that stream.
 *  * Device memory is obtained through the caller's allocator callbacks when
 *    given (e.g. a framework's caching allocator), else cudaMalloc/cudaFree.
 *    The context owns everything it allocates and frees it in sgn_destroy.
 *  * Not thread-safe per context: one host thread drives one context.
 */
#ifndef SGN_H
#define SGN_H

#include <stddef.h>

#ifdef __cplusplus
#define SGN_EXTERN extern "C"
#else
#define SGN_EXTERN extern
#endif
#define SGN_API SGN_EXTERN __attribute__((visibility("default")))

typedef struct sgn_ctx sgn_ctx;

typedef enum {
    SGN_OK = 0,
    SGN_ERR_ARG = 1,            /* invalid argument (size, pointer, range) */
    SGN_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SGN_ERR_NOT_CONVERGED = 3,  /* max_cycles reached; x holds the last iterate */
    SGN_ERR_BREAKDOWN = 4,      /* a shifted Hessenberg system was singular */
    SGN_ERR_DEFLATION = 5,      /* deflation data missing, ambiguous or inaccurate */
    SGN_ERR_NONFINITE = 6,      /* NaN or Inf met in the inputs or the iteration */
    SGN_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
    SGN_ERR_STATE = 8,          /* call order violated (e.g. apply before load_gauge) */
    SGN_ERR_ALLOC = 9           /* device allocation failed */
} sgn_status;

/* Arithmetic of the solve.
 *  SGN_PREC_FP64:  stencil, Krylov basis, coefficients and iterates in FP64.
 *  SGN_PREC_MIXED: stencil and Krylov basis in FP32; inner products, norms,
 *                  Hessenberg matrix, shifted solves, restart coefficients,
 *                  deflation coefficients and iterates in FP64; followed by
 *                  per-shift iterative refinement on the true FP64 residual. */
typedef enum { SGN_PREC_FP64 = 0, SGN_PREC_MIXED = 1 } sgn_precision;

/* Storage of the FP32 stencil's links (mixed form only). */
typedef enum { SGN_LINKS_FP32 = 0, SGN_LINKS_BF16 = 1, SGN_LINKS_FP16 = 2 } sgn_link_storage;

/* Which Krylov space carries the partial fractions (Sec. 2 with eq. (6.2)):
 *  SGN_FORM_A2:  the s systems (A^2 - sigma_i) x_i = A (I - P) b in K(A^2) (default);
 *  SGN_FORM_A:   the same function split as t / (t^2 - sigma) = [(t - a)^{-1} + (t + a)^{-1}] / 2,
 *                a = sqrt(sigma_i) (a = +-i tan(theta_i)/c for eq. (6.2)'s negative shifts):
 *                2s systems (A -+ a_i) x = (I - P) b with weights omega_i / 2 in K(A) --
 *                one stencil per Krylov step instead of two.  FP64 form only. */
typedef enum { SGN_FORM_A2 = 0, SGN_FORM_A = 1 } sgn_formulation;

/* The multishift Krylov method (Sec. 2 and Sec. 4):
 *  SGN_METHOD_FOM:   FOM-LR, Algorithm 1 (default);
 *  SGN_METHOD_GMRES: GMRES-LR, restarted multishift GMRES with LR deflation: the shift of
 *                    smallest modulus (the slowest system) takes the minimal-residual step,
 *                    y_s = argmin ||beta e_1 - (Hbar_k - sigma_s I~) y||, and its residual
 *                    V_{k+1} z restarts the next cycle; every other shift keeps its residual
 *                    collinear by the bordered (k+1) x (k+1) system
 *                    [Hbar_k - sigma_i I~ | z] (y_i, rho_i') = beta rho_i e_1.
 *                    FP64 form of SGN_FORM_A2 only. */
typedef enum { SGN_METHOD_FOM = 0, SGN_METHOD_GMRES = 1 } sgn_method;

/* Flags of sgn_apply. */
#define SGN_APPLY_HOST_BUFFERS 1  /* b and x are host pointers (copied inside the call) */
#define SGN_APPLY_ADJOINT 2       /* apply sign(H_W(-mu)) = sign(H_W(mu))^dag instead */
#define SGN_APPLY_NO_A 4          /* right-hand side of the shifted systems is (I - P) b, not A (I - P) b:
                                     x_shift[i] ~ (A^2 - sigma_i)^{-1} (I - P) b (used by the gradient) */

typedef void* (*sgn_alloc_fn)(size_t bytes, void* user);
typedef void (*sgn_free_fn)(void* ptr, size_t bytes, void* user);

typedef struct {
    int status;           /* sgn_status of the solve */
    int cycles;           /* restart cycles of the multishift phase (max over columns) */
    int matvecs;          /* applications of H_W per column (max over columns) */
    int refine_rounds;    /* mixed form: refinement rounds */
    int refine_cycles;    /* mixed form: restart cycles spent in refinement */
    int breakdown;        /* 1 if some Arnoldi cycle met an invariant subspace */
    double res_est;       /* max over columns and shifts of |rho_i| ||r|| / ||b~|| */
    double err_est;       /* mixed form: estimated relative error of x after refinement */
    double ms;            /* wall time of the call in milliseconds (device events) */
    long long kernels;    /* kernel launches issued by the call (graph nodes counted per replay) */
} sgn_report;

/* Create a context for a lattice of extent dims[4] = {Lx, Ly, Lz, Lt} (each >= 2).
 * alloc/free may be NULL (then cudaMalloc/cudaFree); user is passed through.
 * stream is a cudaStream_t (NULL = legacy default stream).
 * Defaults: mu = 0, m_W = -1.6, antiperiodic in t only, no rational function,
 * k = 40, tol = 1e-10, max_cycles = 1000, projection every cycle (Algorithm 1),
 * FP64 form, no deflation.  Errors: SGN_ERR_ARG, SGN_ERR_CUDA. */
SGN_API int sgn_create(sgn_ctx** out, const int dims[4], sgn_alloc_fn alloc, sgn_free_fn free_,
                       void* user, void* stream);

/* Release everything the context owns.  NULL is accepted. */
SGN_API int sgn_destroy(sgn_ctx* ctx);

/* Change the stream used by later calls. */
SGN_API int sgn_set_stream(sgn_ctx* ctx, void* stream);

/* Copy the gauge field (Sec. 1: the links of D_W) into the context: complex128,
 * [site][dir][3][3]; on_device = 1 for a device pointer, 0 for host memory.
 * The caller keeps ownership of `links`.  Non-finite entries: SGN_ERR_NONFINITE
 * (checked for host links; device links are not read back).  Drops deflation
 * data as sgn_set_mu does. */
SGN_API int sgn_load_gauge(sgn_ctx* ctx, const double* links, int on_device);

/* Quark chemical potential mu: forward time hops carry e^{+mu}, backward e^{-mu}
 * (Sec. 1; non-Hermitian for mu != 0).  A new value drops any deflation data,
 * which belong to one operator (eq. (4.1)).  If there were any, sgn_apply,
 * sgn_apply_shifts, sgn_overlap_apply, sgn_overlap_solve, sgn_apply_direct and
 * sgn_grad_mu then return SGN_ERR_STATE until deflation data are built
 * (sgn_build_deflation), set (sgn_set_deflation), or explicitly cleared
 * (sgn_set_deflation with m = 0).  sgn_load_gauge, sgn_set_kernel_mass and
 * sgn_set_boundary do the same. */
SGN_API int sgn_set_mu(sgn_ctx* ctx, double mu);

/* Wilson kernel mass m_W (the workloads use -1.6).  A new value drops deflation
 * data as sgn_set_mu does. */
SGN_API int sgn_set_kernel_mass(sgn_ctx* ctx, double m_w);

/* Boundary conditions: antiperiodic[nu] = 1 flips the sign of hops that wrap
 * direction nu.  Default {0, 0, 0, 1}.  A change drops deflation data as
 * sgn_set_mu does. */
SGN_API int sgn_set_boundary(sgn_ctx* ctx, const int antiperiodic[4]);

/* Kenney-Laub partial fractions, eq. (6.2), with the scale c of Sec. 6 folded in:
 * sigma[i] = -tan^2(theta_i) / c^2, omega[i] = sec^2(theta_i) / (s c),
 * theta_i = pi (i + 1/2) / (2 s), i = 0..s-1, so that
 * g_s(c t) = t sum_i omega[i] / (t^2 - sigma[i]).  Host arrays of length s.
 * Needs no context.  Errors: SGN_ERR_ARG (s < 1, c <= 0, NULL). */
SGN_API int sgn_kenney_laub(int s, double c, double* sigma, double* omega);

/* Shifts and weights of the rational function applied to A^2, eq. (2.1) read
 * with t^2 (eq. (6.2)): x = A sum_i omega[i] (A^2 - sigma[i])^{-1} (I - P) b.
 * Host arrays of length s, 1 <= s <= 32.  Copied. */
SGN_API int sgn_set_rational(sgn_ctx* ctx, int s, const double* sigma, const double* omega);

/* Restart length k (Algorithm 1's k = k_max, 1 <= k <= 64), stopping tolerance on
 * max_i |rho_i| ||r|| / ||b~|| (eq. (3.1)), cycle cap, and whether the
 * projection step r = (I - P) r runs after every cycle (Algorithm 1; 0 gives
 * the variant without it compared in Fig. 2). */
SGN_API int sgn_set_restart(sgn_ctx* ctx, int k, double tol, int max_cycles, int project_each_cycle);

/* Arithmetic form (sgn_precision) and, for the mixed form, the relative error
 * of x that refinement aims at (e.g. 1e-8).  link_storage (sgn_link_storage)
 * selects the links the FP32 stencil reads: FP32, BF16 or FP16 (all three are
 * rounded from the FP64 field at sgn_load_gauge; the true residuals of the
 * refinement always use the FP32 links).  Errors: SGN_ERR_ARG. */
SGN_API int sgn_set_precision(sgn_ctx* ctx, int precision, double target_rel_err, int link_storage);

/* Krylov space of the partial fractions (sgn_formulation).  SGN_FORM_A needs
 * the FP64 form and has no per-shift output (sgn_apply_shifts, sgn_grad_mu
 * return SGN_ERR_STATE).  Errors: SGN_ERR_ARG. */
SGN_API int sgn_set_formulation(sgn_ctx* ctx, int form);

/* Multishift method (sgn_method).  SGN_METHOD_GMRES with the mixed form or SGN_FORM_A
 * makes sgn_apply return SGN_ERR_STATE.  Errors: SGN_ERR_ARG. */
SGN_API int sgn_set_method(sgn_ctx* ctx, int method);

/* Mixed form only (no counterpart in the paper, which works in FP64): the
 * restart length of the FP32 correction solves that bring each shifted
 * system's true FP64 residual below the tolerance (0: min(k, 16)), and how many
 * shifted systems one correction batch solves side by side (0: up to 10 nrhs,
 * bounded by memory).  Errors: SGN_ERR_ARG (k_refine > 64, max_batch > 4096). */
SGN_API int sgn_set_refinement(sgn_ctx* ctx, int k_refine, int max_batch);

/* LR deflation data of Sec. 4 (eq. (4.1)): m right eigenvectors R and left
 * eigenvectors L (each n x m, column j = one field of n = 12 V complex128,
 * columns back to back), eigenvalues lambda (m complex128), normalised so that
 * L^dag R = I_m.  on_device as in sgn_load_gauge.  Copied; m = 0 clears (and
 * lifts the SGN_ERR_STATE refusal that follows a change of the operator).
 * Errors: SGN_ERR_ARG, SGN_ERR_NONFINITE, SGN_ERR_DEFLATION (Re lambda_j = 0:
 * sign(Re lambda) undefined). */
SGN_API int sgn_set_deflation(sgn_ctx* ctx, int m, const double* R, const double* L,
                              const double* lambda, int on_device);

/* Compute LR deflation data on the GPU (the paper leaves the method open,
 * Sec. 4): the m eigenpairs of H_W(mu) of smallest |lambda| (right vectors from
 * H_W(mu), left vectors from H_W(-mu) = H_W(mu)^dag), biorthonormalised.
 * `extra` further eigenvalues are computed to expose the gap.  eig_tol bounds
 * the relative eigen-residual ||A r - lambda r|| / (|lambda| ||r||).
 * lambda_out (host, 2*(m+extra) doubles, may be NULL) receives the eigenvalues.
 * Errors: SGN_ERR_DEFLATION (no convergence or ambiguous selection). */
SGN_API int sgn_build_deflation(sgn_ctx* ctx, int m, int extra, double eig_tol, double* lambda_out);

/* The next e eigenpairs beyond the deflated ones (right R, left L with
 * L^dag R = I, also biorthogonal to the deflated pairs; lambda: e complex128),
 * in the layout of sgn_set_deflation.  They are not deflated in the solve; the
 * derivative sgn_grad_mu treats them exactly in its reduced resolvents, so that
 * its iterative part works on the spectrum beyond them.  sgn_build_deflation
 * keeps its `extra` pairs here.  e = 0 clears them.  Errors: SGN_ERR_ARG,
 * SGN_ERR_NONFINITE. */
SGN_API int sgn_set_deflation_extra(sgn_ctx* ctx, int e, const double* R, const double* L, const double* lambda,
                                    int on_device);

/* Copy the current deflation data out: R, L (n x m each) and lambda (m), all
 * complex128 host arrays sized by the caller (any may be NULL). */
SGN_API int sgn_get_deflation(sgn_ctx* ctx, int* m, double* R, double* L, double* lambda);

/* Apply the deflated rational sign approximation to nrhs fields (Algorithm 1):
 * x = sign(H_W(mu)) b within the accuracy of eq. (6.2) and the tolerance.
 * b, x: nrhs fields of complex128 each; device pointers unless flags has
 * SGN_APPLY_HOST_BUFFERS.  Each column has its own Krylov space; the columns
 * run in lockstep and share every link load of the stencil.  rep may be NULL.
 * Returns SGN_ERR_NOT_CONVERGED (x holds the last iterate) if max_cycles is hit.
 * Errors: SGN_ERR_STATE (no gauge / rational function, or deflation data dropped
 * by a change of the operator), SGN_ERR_ARG, SGN_ERR_NONFINITE (NaN or Inf in host
 * b, or met in the iteration), SGN_ERR_BREAKDOWN (a shifted Hessenberg system
 * (H_k - sigma_i) was singular: a shift on a Ritz value), SGN_ERR_CUDA. */
SGN_API int sgn_apply(sgn_ctx* ctx, const double* b, double* x, int nrhs, int flags, sgn_report* rep);

/* As sgn_apply, and also return the iterate of every shifted system,
 * x_shift[i] ~ (A^2 - sigma_i)^{-1} A (I - P) b (eq. (2.2) with the A^2 reading):
 * s * nrhs fields, shift-major ([i][rhs]), device pointers. */
SGN_API int sgn_apply_shifts(sgn_ctx* ctx, const double* b, double* x, double* x_shift, int nrhs,
                             int flags, sgn_report* rep);

/* Flags of sgn_hw_apply. */
#define SGN_HW_ADJOINT 1 /* apply H_W(mu)^dag = H_W(-mu) */
#define SGN_HW_PACKED 2  /* in and out are in the packed layout (sgn_pack_fields) */
#define SGN_HW_FLOAT_FLOAT 4 /* with SGN_PREC_FP64: float-float arithmetic on the FP32 units */

/* The Wilson kernel alone (Sec. 1): out = H_W(mu) in (or H_W(-mu) with
 * SGN_HW_ADJOINT) for nrhs fields.  precision SGN_PREC_FP64: complex128 fields;
 * SGN_PREC_MIXED: complex64 fields with the FP32 (or BF16, see
 * sgn_set_precision) links.  Device pointers; in and out must not overlap.
 * Natural-order fields are packed into a staging buffer, the stencil runs on
 * the packed copy and the result is unpacked; with SGN_HW_PACKED the stencil
 * runs on the caller's packed fields directly (no staging, one kernel).
 * SGN_HW_FLOAT_FLOAT (SGN_PREC_FP64 only): complex128 in and out, the stencil in
 * float-float arithmetic (each real a sum of two floats, error-free transforms)
 * on the FP32 units, within about 1e-13 of the FP64 stencil; the mixed form
 * forms its true residuals this way.
 * Errors: SGN_ERR_ARG (unknown precision or flag, SGN_HW_FLOAT_FLOAT with the
 * mixed precision), SGN_ERR_STATE (no gauge). */
SGN_API int sgn_hw_apply(sgn_ctx* ctx, const void* in, void* out, int nrhs, int precision, int flags);

/* The overlap operator built on the sign function (Sec. 1):
 *   y = D_ov b = b + gamma5 F(A) b,
 * F(A) the deflated rational sign function sgn_apply computes (same settings:
 * precision, deflation, tolerance).  b, y: nrhs complex128 device fields, natural
 * order, not overlapping.  Errors: SGN_ERR_STATE (no gauge / rational function). */
SGN_API int sgn_overlap_apply(sgn_ctx* ctx, const double* b, double* y, int nrhs);

/* x = D_ov^{-1} b by restarted GMRES(k) from x = 0, every Arnoldi step one batched
 * sign solve over the nrhs columns; stops when every column has
 * ||b - D_ov x|| <= tol ||b|| (checked on the true residual at each restart) or after
 * max_restarts restarts.  iterations (may be NULL): applications of D_ov in the Arnoldi
 * steps; relres (may be NULL): the worst column's final relative residual.  The inner
 * solves' tolerance (sgn_set_restart) should be well below tol.  b, x: device fields.
 * Errors: SGN_ERR_ARG (k outside 1..64), SGN_ERR_NOT_CONVERGED (x holds the last iterate). */
SGN_API int sgn_overlap_solve(sgn_ctx* ctx, const double* b, double* x, int nrhs, double tol, int k,
                              int max_restarts, int* iterations, double* relres);

/* The direct projection the paper compares Algorithm 1 with (Sec. 6, eq. (6.3)):
 *   x = x_P + ||r|| V_k sign(H_k) e_1,   r = (I - P) b,   x_P = R sign(Re Lambda) L^dag b,
 * V_k, H_k from k steps of Arnoldi on A = H_W(mu) itself started at r (two classical
 * Gram-Schmidt passes, FP64), sign(H_k) by Roberts' Newton iteration
 * X <- (X + X^{-1}) / 2 on the host.  No rational approximation and no restarts: the
 * k + 1 basis fields per column stay in device memory, and the Newton step costs
 * O(k^3) per column.  Uses the deflation set up by sgn_build_deflation or
 * sgn_set_deflation (none when m = 0); ignores the rational function, precision and
 * tolerance settings.  flags: 0 or SGN_APPLY_ADJOINT (A^dag = H_W(-mu)).  b, x: nrhs
 * complex128 device fields, natural order, not overlapping.  k_used (may be NULL):
 * the largest Krylov dimension used, below k only when an invariant subspace was
 * found (where the projection is exact).  Errors: SGN_ERR_ARG (k outside 1..4096,
 * unknown flag), SGN_ERR_STATE (no gauge), SGN_ERR_NOT_CONVERGED (the Newton
 * iteration met a singular iterate: a Ritz value on the imaginary axis). */
SGN_API int sgn_apply_direct(sgn_ctx* ctx, const double* b, double* x, int nrhs, int k, int flags, int* k_used);

/* Layout conversion of nfield fields between the natural order
 * [site][spin][colour] and the packed order the library keeps internally:
 * complex entry k = 3 spin + colour of site s at (k/2) * 2V + 2s + (k mod 2)
 * within its field (six planes of two entries per site, so a warp's loads of
 * consecutive sites are contiguous).  Device pointers, in != out;
 * precision SGN_PREC_FP64 (complex128) or SGN_PREC_MIXED (complex64);
 * 1 <= nfield <= 65535.  Every other call of this interface takes and returns
 * natural-order fields. */
SGN_API int sgn_pack_fields(sgn_ctx* ctx, const void* in, void* out, int nfield, int precision);
SGN_API int sgn_unpack_fields(sgn_ctx* ctx, const void* in, void* out, int nfield, int precision);

/* Inner products out[c*J + j] = <V_j, w_c> = V_j^dag w_c of J fields V (one basis
 * shared by every column) with nrhs fields w -- the coefficients of classical
 * Gram-Schmidt (V^dag w, eq. (2.4)) and of the projection step (L^dag r, eq. (4.5)).
 * V: J complex128 device fields back to back; w: nrhs complex128 device fields;
 * out: host array of nrhs*J complex128.  1 <= J <= 64.  FP64 accumulation in a
 * fixed order (deterministic).  Scratch for the per-block partial sums comes from
 * the context's allocator and is kept for later calls. */
SGN_API int sgn_inner_products(sgn_ctx* ctx, const double* V, int J, const double* w, int nrhs, double* out);

/* The inner products of sgn_inner_products, for callers that cannot allocate
 * device memory: applications whose framework owns every device allocation (a
 * fixed arena sized up front, where an outside cudaMalloc is forbidden or would
 * exceed the budget), and latency-critical loops that must not pay for
 * cudaMalloc/cudaFree, which can synchronise the device.  (The paper has no
 * counterpart; this is a deployment variant of the Gram-Schmidt and projection
 * inner products above.)
 *   V: J complex128 device fields of n complex numbers each, back to back;
 *   w: nrhs complex128 device fields; out: DEVICE array of nrhs*J complex128,
 *   out[c*J + j] = V_j^dag w_c.  n even, 1 <= J <= 64, 1 <= nrhs <= 512.
 * No context and no allocation: the per-block partial sums live in one fixed
 * 8 MiB device array inside the library (held on every device that loads the
 * library until the process exits).  The call is rejected (SGN_ERR_ARG) when
 * nrhs * J * ceil(n / 1024) * 16 bytes exceeds 8 MiB.  The first call on a device
 * looks up the array's device address (with that device current) and keeps it
 * for the life of the process; make that first call before any stream capture.
 * A device reset (cudaDeviceReset) reloads the library's device code and makes
 * the kept address stale: do not use this entry point after resetting a device.
 * All calls share the array and each call clears the part that must start at
 * zero: calls that overlap on the GPU (other streams or threads) race and must
 * be serialised by the caller.  Work is queued on `stream` (a cudaStream_t); the
 * call does not synchronise. */
SGN_API int sgn_inner_products_noalloc(const double* V, int J, const double* w, long long n, int nrhs, double* out,
                                       void* stream);

/* dH_W/dmu applied to nrhs complex128 device fields: out = gamma5 dD_W/dmu in,
 * dD_W/dmu psi(x) = -1/2 [(1 - gamma_t) e^{+mu} U_t(x) psi(x+t) - (1 + gamma_t) e^{-mu} U_t(x-t)^dag psi(x-t)]
 * (only the time hops of D_W(mu) depend on mu, Sec. 1). */
SGN_API int sgn_dhw_dmu_apply(sgn_ctx* ctx, const double* in, double* out, int nrhs);

/* Derivative with respect to mu of the loss Re<g, x(mu)>, x = F(A) b the deflated
 * rational sign function this context applies (Sec. 4, eq. (6.2)),
 * F(A) = R S L^dag + G(A)(I - P), G(A) = sum_i omega_i (A^2 - sigma_i)^{-1} A,
 * A = H_W(mu), A' = dH_W/dmu, per column:
 *   dmu[c] = Re [ sum_i omega_i < z_i, A' v - A' A x_i - A A' x_i >        (v = (I - P) b)
 *               - sum_j (l_j^dag b) < S_j^dag (s_j g - G(A)^dag g), A' r_j >
 *               - sum_j (s_j - g(lambda_j)) <g, r_j> l_j^dag A' S_j b ],
 * x_i = (A^2 - sigma_i)^{-1} A v, z_i = (A^dag^2 - sigma_i)^{-1} g, s_j = sign(Re lambda_j),
 * S_j = (A - lambda_j)^{-1}(I - r_j l_j^dag) (the eigenvector motion of the
 * deflated pairs; the deflation data must be the eigenpairs at this mu).  The
 * reduced resolvents come from multishift solves with the complex shifts
 * lambda_j^2.  With m = 0 only the first sum remains.
 * b, g: nrhs complex128 device fields; dmu: host array of nrhs doubles. */
SGN_API int sgn_grad_mu(sgn_ctx* ctx, const double* b, const double* g, int nrhs, double* dmu);

/* Diagnostic: the Hessenberg matrix H_k of the Arnoldi relation (eq. (2.4)) on A^2,
 * as the last restart cycle of the last FP64-form sgn_apply / sgn_apply_shifts of
 * this context left it, for column `col`: H receives (k+1) x k complex128 entries,
 * row-major (entry (i, j) at 2 (i k + j)), k the restart length of that solve;
 * k_used (may be NULL) the Arnoldi steps that cycle took (below k after an
 * invariant subspace).  At mu = 0, A^2 is Hermitian and H_k is tridiagonal up to
 * rounding (the Lanczos case of Sec. 2).  Synchronises the stream.
 * Errors: SGN_ERR_STATE (no FP64-form solve yet), SGN_ERR_ARG. */
SGN_API int sgn_get_hessenberg(sgn_ctx* ctx, int col, double* H, int* k_used);

/* Kernel timing (observability).  With on = 1, later solves record CUDA events
 * around every launch of the restart cycle's main kernels, inside the captured
 * graph, and accumulate per class: 0 = Wilson stencil, 1 = fused Gram-Schmidt
 * reduction (k_dcgs_dots), 2 = fused Gram-Schmidt update (k_dcgs_update),
 * 3 = second stage of those reductions with the step's scalar work (k_reduce),
 * 4 = per-shift update x_i += V y_i (k_update_shifts).
 * Each event pair brackets one launch on the solver's stream.  Switching on or
 * off resets the totals. */
SGN_API int sgn_set_kernel_timing(sgn_ctx* ctx, int on);

/* Totals of class `cls` since timing was switched on: summed milliseconds,
 * launches, and algorithmic bytes (each input field read once, each output
 * field written once; only the columns not yet converged when the cycle
 * started count, since converged columns skip their work). */
SGN_API int sgn_get_kernel_timing(sgn_ctx* ctx, int cls, double* ms, long long* launches, double* bytes);

/* Thread-local message for the last failing call of this thread. */
SGN_API const char* sgn_last_error(void);

/* Library version string. */
SGN_API const char* sgn_version(void);

#endif /* SGN_H */
