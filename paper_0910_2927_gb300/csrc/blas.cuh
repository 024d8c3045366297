// Tall-skinny vector kernels for the Arnoldi process (eq. (2.4)), the update
// of Algorithm 1 and the LR projection (Sec. 4).  Declarations.
#pragma once

#include "sgn_internal.cuh"

namespace sgn {

// Per-column solver state kept on the device, so that one restart cycle is a
// fixed sequence of launches with no host round trip (captured as a graph).
struct DevState {
    double2* H;        // [col][(kmax+1) * kmax] Hessenberg matrix, row-major (row i, col j)
    double2* red;      // [col][rstride] reduction results / coefficients of the next pass
    double2* h1;       // [col][rstride] first Gram-Schmidt coefficients of the current step
    double2* coef;     // [col][rstride] combined update coefficients sum_i omega_i y_i
    double2* y;        // [col][s][kmax] shifted solutions of the current cycle
    double2* rho;      // [col][s] collinearity factors (eq. (3.1))
    double* norm0;     // [col] ||A^2 v_j|| before orthogonalisation
    double* scale;     // [col] scale applied by the next normalising pass
    double* beta;      // [col] ||r|| of the restart vector
    double* bnorm;     // [col] ||b~||
    double* resest;    // [col] max_i |rho_i| ||r|| / ||b~||
    const double* sigma;  // [col][s] shifts (per column: the mixed refinement solves one shift per column)
    const double* omega;  // [col][s] weights
    const double* sigma_im = nullptr;  // [col][s] imaginary parts of the shifts (null: real shifts)
    double2* gres = nullptr;  // [col][kmax + 1] minimal-residual form: coefficients of the new residual in V_{k+1}
    int* kk;           // [col] Krylov dimension of the current cycle
    int* done;         // [col] converged (column work is skipped)
    int* skip;         // [col] done or broken down in this cycle
    int* err;          // [1] device error word (bit 0: singular shifted system; bit 1: non-finite)
    // Optional (both or neither): per-slot sums and per-column arrival counters for the
    // split second-stage reduction (several CTAs per column, the last one does the
    // column's scalar work).  Null: one CTA per column.
    double2* sums = nullptr;  // [col][rstride]
    int* rcount = nullptr;    // [col], zero between launches
    int kmax;
    int s;
    int rstride;
    double tol;
    double bd_tol;     // breakdown threshold relative to norm0
};

enum ReduceMode {
    RM_STORE = 0,        // red[col][j] = sum_j
    RM_H1 = 1,           // h1[col][j] = sum_j (j < J), norm0 = sqrt(sum_J)
    RM_P2 = 2,           // second CGS pass: Hessenberg column, h_{j+1,j}, breakdown, scale
    RM_BETA_FIRST = 3,   // bnorm = beta = sqrt(sum_0), rho = 1, scale = 1/beta
    RM_BETA_RESTART = 4, // beta = sqrt(sum_0), residual estimate, convergence, scale = 1/beta
    RM_SIGNED = 5,       // red[col][j] = sign(Re lambda_j) * sum_j (x_P coefficients)
    RM_DCGS = 6,         // delayed CGS2 step j: rho, column j-1 correction, tentative column j, update coefficients
    RM_DCGS_FINAL = 7    // delayed CGS2 closing pass of a cycle (no new candidate)
};

template <class T>
cudaError_t mdot(Basis<T> V, int J, const T* w, int64_t wsr, int64_t n, int ncol, const Reduce& rd,
                 int with_norm, const int* skip, cudaStream_t st);
cudaError_t reduce(const Reduce& rd, int nslot, int ncol, int mode, int colidx, const DevState& S,
                   const double2* lambda, cudaStream_t st);
template <class T>
cudaError_t maxpy_mdot(Basis<T> V, int J, const double2* coef, int cstride, T* w, int64_t wsr, int64_t n,
                       int ncol, const Reduce& rd, const int* skip, cudaStream_t st);
template <class T>
cudaError_t maxpy_scale(Basis<T> V, int J, const double2* coef, int cstride, const T* w, int64_t wsr, T* out,
                        int64_t osr, const double* scale, int64_t n, int ncol, const int* skip, cudaStream_t st);
template <class T>
cudaError_t update_x(Basis<T> V, int J, const double2* coef, int cstride, double2* x, int64_t xsr, int64_t n,
                     int ncol, const int* skip, const int* kk, cudaStream_t st);
template <class T>
cudaError_t update_shifts(Basis<T> V, int J, const double2* y, int s, int kmax, double2* xs, int64_t xs_shift,
                          int64_t xs_col, int64_t n, int ncol, const int* skip, const int* kk, cudaStream_t st);

// Delayed CGS2 (one fused reduction and one fused update per Arnoldi step).
template <class T>
cudaError_t dcgs_dots(Basis<T> V, int J, const T* u, const T* z, int64_t wsr, int64_t n, int ncol, const Reduce& rd,
                      const int* skip, cudaStream_t st);
template <class T>
cudaError_t dcgs_update(Basis<T> V, int J, const double2* coef, int cstride, T* u, const T* z, T* next, int64_t wsr,
                        int64_t n, int ncol, const int* skip, cudaStream_t st);

// out = a x + b y + c z over `count` complex elements (z may be null).
template <class T>
cudaError_t axpby3(T* out, double a, const T* x, double b, const T* y, double c, const T* z, int64_t count,
                   cudaStream_t st);
// Z_j = sum_i C[i][j] Y_i for q input and r output fields of n complex (C: device, row-major q x r).
template <class T>
cudaError_t block_combine(const T* Y, int q, const double2* C, int r, T* Z, int64_t n, cudaStream_t st);
// Seeded complex Gaussian entries (counter-based, SplitMix64 + Box-Muller).
template <class T>
cudaError_t random_fill(T* out, int64_t count, uint64_t seed, cudaStream_t st);

// Type conversions of whole fields.
cudaError_t convert_f64_to_f32(const double2* in, float2* out, int64_t count, cudaStream_t st);
cudaError_t convert_f32_to_f64(const float2* in, double2* out, int64_t count, cudaStream_t st);
cudaError_t links_f64_to_bf16(const double2* in, __nv_bfloat162* out, int64_t count, cudaStream_t st);
cudaError_t links_f64_to_f16(const double2* in, __half2* out, int64_t count, cudaStream_t st);

// Small dense steps (hess.cu).  prepare_small_kernels sets launch attributes once
// per device (before any stream capture).
cudaError_t prepare_small_kernels();
cudaError_t shifted_solves(const DevState& S, int ncol, cudaStream_t st);
// Minimal-residual (GMRES) form for one shift per column: y, rho = 1 and the new
// residual's coefficients in S.gres (k_shifted_lsq).
cudaError_t shifted_lsq(const DevState& S, int ncol, cudaStream_t st);
cudaError_t combine_shifts(const DevState& S, int ncol, cudaStream_t st);

// y = a + beta gamma5 s for nfield packed complex128 fields (gamma5: spins 2, 3 negated).
cudaError_t gamma5_axpy(double2* y, const double2* a, const double2* s, double beta, int64_t vol, int nfield,
                        cudaStream_t st);

// Refinement residual update r_j += sigma_j d_j - w_j (w_j = A^2 d_j in FP32) for nb
// systems: r_j at r + roff[j], w_j and d_j at j * n.
cudaError_t correct_residuals(double2* r, const long long* roff, const double* sig, const float2* w,
                              const double2* d, int64_t n, int nb, cudaStream_t st);

// Tall-skinny products of a basis V (J <= 64 fields, stride sv) with N columns W
// (complex128, stride sw): tsmm_tn writes the partials of V^dag W into rd (then
// reduce(rd, J, N, RM_STORE, ...) gives red[col * rstride + j]); tsmm_nn does
// W_col += alpha sum_j V_j C[col * cstride + j].  FP32 products, FP64 sums over CTAs.
template <class TV>
cudaError_t tsmm_tn(const TV* V, int64_t sv, int J, const double2* W, int64_t sw, int N, int64_t n,
                    const Reduce& rd, cudaStream_t st);
template <class TV>
cudaError_t tsmm_nn(const TV* V, int64_t sv, int J, const double2* C, int cstride, double2* W, int64_t sw, int N,
                    int64_t n, double alpha, cudaStream_t st);

// Number of blocks per column used by the reductions for n complex elements.
template <class T>
int reduce_blocks(int64_t n);
// CTAs per column for a grid of ncol columns that fills whole waves (1, 2 or 4
// packs per thread); a Reduce built with it serves every kernel of the file.
template <class T>
int wave_blocks(int64_t n, int ncol);

}  // namespace sgn
