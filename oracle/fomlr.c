/*
 * Oracle: Kenney-Laub partial fractions and restarted FOM-LR(m,k).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * What is computed (the A^2 reading of eq. (6.2) combined with Algorithm 1):
 *
 *   x = R sign(Re Lambda) L^dag b  +  sum_i omega_i (A^2 - sigma_i)^{-1} A (I - P) b,
 *
 * P = R L^dag, with sigma_i, omega_i from eq. (6.2) and the scale c of
 * Sec. 6 folded in (sigma_i / c^2, omega_i / c).  The s shifted systems of
 * eq. (2.2) are therefore systems in A^2 with the common right-hand side
 * b~ = A (I - P) b, and Algorithm 1 runs on A^2 with b~ as its first
 * restart vector.  Each Arnoldi step orthogonalises by classical Gram-Schmidt
 * applied twice; the shifted Hessenberg systems are solved by Gaussian
 * elimination with partial pivoting.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* eq. (6.2): g_s(t) = t sum_i omega_i / (t^2 - sigma_i),
 *   omega_i = (1/s) cos^{-2}(theta_i), sigma_i = -tan^2(theta_i),
 *   theta_i = (pi / 2s)(i - 1/2), i = 1..s.
 * Sec. 6 uses g_s(c t); c t sum omega_i / (c^2 t^2 - sigma_i) equals
 * t sum (omega_i / c) / (t^2 - sigma_i / c^2), which is what is returned. */
int orc_kenney_laub(int s, double c, double* sigma, double* omega) {
    if (s < 1 || !(c > 0)) return 1;
    for (int i = 1; i <= s; ++i) {
        double th = M_PI / (2.0 * s) * (i - 0.5);
        double t = tan(th), co = cos(th);
        sigma[i - 1] = -(t * t) / (c * c);
        omega[i - 1] = 1.0 / (s * co * co) / c;
    }
    return 0;
}

/* ---- plain vector helpers ------------------------------------------------ */

static orc_c dotc(int64_t n, const orc_c* a, const orc_c* b) {  /* a^dag b */
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        orc_c p = conj(a[e]) * b[e];
        re += creal(p);
        im += cimag(p);
    }
    return re + I * im;
}

static double norm2(int64_t n, const orc_c* a) { return sqrt(creal(dotc(n, a, a))); }

static void axpy(int64_t n, orc_c alpha, const orc_c* xv, orc_c* yv) {  /* y += alpha x */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) yv[e] += alpha * xv[e];
}

static void scal_copy(int64_t n, orc_c alpha, const orc_c* xv, orc_c* yv) {  /* y = alpha x */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) yv[e] = alpha * xv[e];
}

/* ---- deflation: Sec. 4, eqs. (4.2)-(4.5) --------------------------------- */

/* c = L^dag v (m coefficients) */
static void ldag(int64_t n, int m, const orc_c* L, const orc_c* v, orc_c* c) {
    for (int j = 0; j < m; ++j) c[j] = dotc(n, L + (int64_t)j * n, v);
}

/* v <- (I - P) v = v - R (L^dag v): the projection step of Algorithm 1 */
static void project(int64_t n, int m, const orc_c* R, const orc_c* L, orc_c* v, orc_c* work) {
    if (m == 0) return;
    ldag(n, m, L, v, work);
    for (int j = 0; j < m; ++j) axpy(n, -work[j], R + (int64_t)j * n, v);
}

/* ---- shifted Hessenberg solve -------------------------------------------- */

/* Solve (H_kk - sigma I) y = rhs0 * e_1 by Gaussian elimination with partial
 * pivoting on the dense kk x kk matrix; H is (k+1) x k, row-major with
 * leading dimension k.  Pivot: the entry of largest modulus, first one on ties. */
static int shifted_solve(int kk, int k, const orc_c* H, double sigma, orc_c rhs0, orc_c* y, orc_c* M) {
    for (int i = 0; i < kk; ++i) {
        for (int j = 0; j < kk; ++j) M[i * kk + j] = H[i * k + j];
        M[i * kk + i] -= sigma;
        y[i] = (i == 0) ? rhs0 : 0;
    }
    for (int j = 0; j < kk; ++j) {
        int p = j;
        for (int i = j + 1; i < kk; ++i)
            if (cabs(M[i * kk + j]) > cabs(M[p * kk + j])) p = i;
        if (M[p * kk + j] == 0) return 1;
        if (p != j) {
            for (int l = 0; l < kk; ++l) {
                orc_c t = M[j * kk + l];
                M[j * kk + l] = M[p * kk + l];
                M[p * kk + l] = t;
            }
            orc_c t = y[j];
            y[j] = y[p];
            y[p] = t;
        }
        for (int i = j + 1; i < kk; ++i) {
            orc_c f = M[i * kk + j] / M[j * kk + j];
            if (f == 0) continue;
            for (int l = j; l < kk; ++l) M[i * kk + l] -= f * M[j * kk + l];
            y[i] -= f * y[j];
        }
    }
    for (int i = kk - 1; i >= 0; --i) {
        orc_c acc = y[i];
        for (int l = i + 1; l < kk; ++l) acc -= M[i * kk + l] * y[l];
        y[i] = acc / M[i * kk + i];
    }
    return 0;
}

/* ---- Algorithm 1 ----------------------------------------------------------- */

int orc_fom_lr(const orc_lattice* lat, const orc_c* U,
               int s, const double* sigma, const double* omega,
               int k, double tol, int max_cycles, int project_each_cycle,
               int m, const orc_c* R, const orc_c* L, const orc_c* lambda,
               const orc_c* b, orc_c* x, orc_c* x_shift, orc_report* rep) {
    const int64_t n = 12LL * lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
    if (s < 1 || k < 1 || m < 0) return 1;

    orc_c* V = malloc(sizeof(orc_c) * n * (k + 1));
    orc_c* w = malloc(sizeof(orc_c) * n);
    orc_c* t = malloc(sizeof(orc_c) * n);
    orc_c* r = malloc(sizeof(orc_c) * n);
    orc_c* H = calloc((size_t)(k + 1) * k, sizeof(orc_c));
    orc_c* h1 = malloc(sizeof(orc_c) * (k + 1));
    orc_c* h2 = malloc(sizeof(orc_c) * (k + 1));
    orc_c* cm = malloc(sizeof(orc_c) * (m > 0 ? m : 1));
    orc_c* y = malloc(sizeof(orc_c) * k);
    orc_c* M = malloc(sizeof(orc_c) * k * k);
    orc_c* rho = malloc(sizeof(orc_c) * s);
    int status = 0;
    if (!V || !w || !t || !r || !H || !h1 || !h2 || !cm || !y || !M || !rho) { status = 2; goto done; }

    orc_report rp = {0, 0, 0, 0, 0.0};

    /* x = x_P = R f(Lambda) L^dag b, f = sign(Re lambda): eq. (4.3) */
    memset(x, 0, sizeof(orc_c) * n);
    if (x_shift) memset(x_shift, 0, sizeof(orc_c) * n * s);
    memcpy(r, b, sizeof(orc_c) * n);
    if (m > 0) {
        ldag(n, m, L, b, cm);
        for (int j = 0; j < m; ++j) {
            double sg = (creal(lambda[j]) > 0) ? 1.0 : -1.0;
            axpy(n, sg * cm[j], R + (int64_t)j * n, x);
            /* r = (I - P) b, eq. (4.2) */
            axpy(n, -cm[j], R + (int64_t)j * n, r);
        }
    }
    /* b~ = A (I - P) b: right-hand side of the shifted systems in A^2 */
    orc_hw(lat, U, r, t);
    memcpy(r, t, sizeof(orc_c) * n);
    rp.matvecs += 1;
    const double bnorm = norm2(n, r);
    for (int i = 0; i < s; ++i) rho[i] = 1.0;
    if (bnorm == 0) { rp.converged = 1; goto finish; }

    for (int cyc = 0; cyc < max_cycles; ++cyc) {
        double beta = norm2(n, r);
        if (beta == 0) { rp.converged = 1; break; }
        scal_copy(n, 1.0 / beta, r, V);
        memset(H, 0, sizeof(orc_c) * (k + 1) * k);
        int kk = k, broke = 0;
        /* k steps of Arnoldi with A^2, eq. (2.4) */
        for (int j = 0; j < k; ++j) {
            orc_hw(lat, U, V + (int64_t)j * n, t);
            orc_hw(lat, U, t, w);
            rp.matvecs += 2;
            double w0 = norm2(n, w);
            for (int l = 0; l <= j; ++l) h1[l] = dotc(n, V + (int64_t)l * n, w);
            for (int l = 0; l <= j; ++l) axpy(n, -h1[l], V + (int64_t)l * n, w);
            for (int l = 0; l <= j; ++l) h2[l] = dotc(n, V + (int64_t)l * n, w);
            for (int l = 0; l <= j; ++l) axpy(n, -h2[l], V + (int64_t)l * n, w);
            for (int l = 0; l <= j; ++l) H[l * k + j] = h1[l] + h2[l];
            double hn = norm2(n, w);
            H[(j + 1) * k + j] = hn;
            if (hn <= 1e-14 * w0) { kk = j + 1; broke = 1; break; }
            scal_copy(n, 1.0 / hn, w, V + (int64_t)(j + 1) * n);
        }
        /* y_i = beta rho_i (H_k - sigma_i I)^{-1} e_1 and the update of x */
        double resmax = 0;
        for (int i = 0; i < s; ++i) {
            if (shifted_solve(kk, k, H, sigma[i], beta * rho[i], y, M)) { status = 4; goto finish; }
            for (int l = 0; l < kk; ++l) {
                axpy(n, omega[i] * y[l], V + (int64_t)l * n, x);
                if (x_shift) axpy(n, y[l], V + (int64_t)l * n, x_shift + (int64_t)i * n);
            }
            /* rho_i = -h_{k+1,k} e_k^T y_i, eq. (3.1) */
            rho[i] = broke ? 0 : -H[kk * k + (kk - 1)] * y[kk - 1];
        }
        rp.cycles = cyc + 1;
        if (broke) { rp.breakdown = 1; rp.converged = 1; rp.res_est = 0; break; }
        memcpy(r, V + (int64_t)kk * n, sizeof(orc_c) * n);   /* r = v_{k+1} */
        if (project_each_cycle) project(n, m, R, L, r, cm);   /* projection step, eq. (4.5) */
        double rn = norm2(n, r);
        for (int i = 0; i < s; ++i) {
            double e = cabs(rho[i]) * rn / bnorm;
            if (e > resmax) resmax = e;
        }
        rp.res_est = resmax;
        if (resmax <= tol) { rp.converged = 1; break; }
    }

finish:
    if (rep) *rep = rp;
    if (status == 0 && !rp.converged) status = 3;
done:
    free(V); free(w); free(t); free(r); free(H); free(h1); free(h2);
    free(cm); free(y); free(M); free(rho);
    return status;
}
