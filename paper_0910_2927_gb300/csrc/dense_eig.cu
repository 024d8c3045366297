// Host-side dense eigensolver for the small Rayleigh-Ritz matrices of the
// deflation set-up (q x q, q <= 96): Householder reduction to upper Hessenberg
// form, shifted QR iteration with Givens rotations (Wilkinson shift) to the
// complex Schur form T = Q^dag G Q, eigenvectors of T by back substitution,
// mapped back through Q.  Textbook algorithm (Golub & Van Loan, Ch. 7).
#include "dense_eig.h"

#include <algorithm>
#include <cmath>

namespace sgn {

using cd = std::complex<double>;

namespace {

inline double abs1(cd z) { return std::abs(z.real()) + std::abs(z.imag()); }

// G <- Q^dag G Q with G upper Hessenberg on exit; Q accumulated (row-major n x n).
void hessenberg(int n, std::vector<cd>& G, std::vector<cd>& Q) {
    auto A = [&](int i, int j) -> cd& { return G[(size_t)i * n + j]; };
    auto Qm = [&](int i, int j) -> cd& { return Q[(size_t)i * n + j]; };
    std::vector<cd> v(n);
    for (int k = 0; k + 2 < n + 0 && k < n - 2; ++k) {
        double alpha = 0;
        for (int i = k + 1; i < n; ++i) alpha += std::norm(A(i, k));
        alpha = std::sqrt(alpha);
        if (alpha == 0) continue;
        cd x0 = A(k + 1, k);
        cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1, 0);
        // v = x + ph * alpha * e1, H = I - 2 v v^dag / (v^dag v)
        for (int i = 0; i < n; ++i) v[i] = 0;
        for (int i = k + 1; i < n; ++i) v[i] = A(i, k);
        v[k + 1] += ph * alpha;
        double vv = 0;
        for (int i = k + 1; i < n; ++i) vv += std::norm(v[i]);
        if (vv == 0) continue;
        // left: G <- H G
        for (int j = 0; j < n; ++j) {
            cd s = 0;
            for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * A(i, j);
            s *= 2.0 / vv;
            for (int i = k + 1; i < n; ++i) A(i, j) -= v[i] * s;
        }
        // right: G <- G H
        for (int i = 0; i < n; ++i) {
            cd s = 0;
            for (int j = k + 1; j < n; ++j) s += A(i, j) * v[j];
            s *= 2.0 / vv;
            for (int j = k + 1; j < n; ++j) A(i, j) -= s * std::conj(v[j]);
        }
        // Q <- Q H
        for (int i = 0; i < n; ++i) {
            cd s = 0;
            for (int j = k + 1; j < n; ++j) s += Qm(i, j) * v[j];
            s *= 2.0 / vv;
            for (int j = k + 1; j < n; ++j) Qm(i, j) -= s * std::conj(v[j]);
        }
        for (int i = k + 2; i < n; ++i) A(i, k) = 0;
    }
}

// Givens rotation [c s; -conj(s) c] (c real) with [c s; -s* c] [a; b] = [r; 0].
void givens(cd a, cd b, double& c, cd& s) {
    double na = std::abs(a), nb = std::abs(b);
    if (nb == 0) {
        c = 1;
        s = 0;
        return;
    }
    if (na == 0) {
        c = 0;
        s = std::conj(b) / nb;
        return;
    }
    double r = std::hypot(na, nb);
    c = na / r;
    s = (a / na) * std::conj(b) / r;
}

}  // namespace

namespace {
// Complex Schur form G = Q T Q^dag (T, Q row-major).  Returns 0 on success.
int schur(int n, const std::vector<cd>& G_in, std::vector<cd>& T, std::vector<cd>& Q, double& norm, int max_iter);
}  // namespace

int dense_eig(int n, const std::vector<cd>& G_in, std::vector<cd>& w, std::vector<cd>& X, int max_iter) {
    std::vector<cd> T, Q;
    double norm = 0;
    if (schur(n, G_in, T, Q, norm, max_iter)) return 1;
    auto A = [&](int i, int j) -> cd& { return T[(size_t)i * n + j]; };
    const double eps = 2.220446049250313e-16;
    // eigenvalues and eigenvectors of the triangular T
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A(i, i);
    std::vector<cd> V((size_t)n * n, 0.0);
    const double small = eps * std::max(norm, 1e-300);
    for (int k = 0; k < n; ++k) {
        V[(size_t)k * n + k] = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            cd s = 0;
            for (int j = i + 1; j <= k; ++j) s += A(i, j) * V[(size_t)j * n + k];
            cd den = A(i, i) - w[k];
            if (std::abs(den) < small) den = small;
            V[(size_t)i * n + k] = -s / den;
        }
    }
    X.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            cd s = 0;
            for (int j = 0; j <= k; ++j) s += Q[(size_t)i * n + j] * V[(size_t)j * n + k];
            X[(size_t)i * n + k] = s;
        }
    for (int k = 0; k < n; ++k) {
        double nr = 0;
        for (int i = 0; i < n; ++i) nr += std::norm(X[(size_t)i * n + k]);
        nr = std::sqrt(nr);
        if (nr > 0)
            for (int i = 0; i < n; ++i) X[(size_t)i * n + k] /= nr;
    }
    return 0;
}

int herm_eig(int n, const std::vector<cd>& G, std::vector<double>& w, std::vector<cd>& X) {
    std::vector<cd> T;
    double norm = 0;
    if (schur(n, G, T, X, norm, 60)) return 1;
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = T[(size_t)i * n + i].real();
    return 0;
}

namespace {
int schur(int n, const std::vector<cd>& G_in, std::vector<cd>& T, std::vector<cd>& Q, double& norm, int max_iter) {
    T = G_in;
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    auto A = [&](int i, int j) -> cd& { return T[(size_t)i * n + j]; };
    if (n > 2) hessenberg(n, T, Q);
    norm = 0;
    for (auto& z : T) norm = std::max(norm, std::abs(z));
    const double eps = 2.220446049250313e-16;
    // shifted QR on the active window [lo, hi]
    int hi = n - 1, iter = 0, total = 0;
    while (hi > 0) {
        // find lo: smallest index with negligible subdiagonal above it
        int lo = hi;
        while (lo > 0) {
            double s = abs1(A(lo - 1, lo - 1)) + abs1(A(lo, lo));
            if (s == 0) s = norm;
            if (abs1(A(lo, lo - 1)) <= eps * s) {
                A(lo, lo - 1) = 0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            --hi;
            iter = 0;
            continue;
        }
        if (++total > max_iter * n) return 1;
        ++iter;
        // Wilkinson shift from the trailing 2x2 block
        cd a = A(hi - 1, hi - 1), b = A(hi - 1, hi), c = A(hi, hi - 1), d = A(hi, hi);
        cd tr = a + d, det = a * d - b * c;
        cd disc = std::sqrt(tr * tr - 4.0 * det);
        cd l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        cd mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (iter % 11 == 10) mu = d + cd(abs1(A(hi, hi - 1)), 0);  // exceptional shift
        // implicit single-shift QR sweep by Givens rotations (bulge chase)
        cd x = A(lo, lo) - mu, y = A(lo + 1, lo);
        for (int k = lo; k < hi; ++k) {
            double cs;
            cd sn;
            givens(x, y, cs, sn);
            // rows k, k+1
            for (int j = (k > lo ? k - 1 : lo); j < n; ++j) {
                cd t1 = A(k, j), t2 = A(k + 1, j);
                A(k, j) = cs * t1 + sn * t2;
                A(k + 1, j) = -std::conj(sn) * t1 + cs * t2;
            }
            // columns k, k+1
            int imax = std::min(hi, k + 2);
            for (int i = 0; i <= imax; ++i) {
                cd t1 = A(i, k), t2 = A(i, k + 1);
                A(i, k) = cs * t1 + std::conj(sn) * t2;
                A(i, k + 1) = -sn * t1 + cs * t2;
            }
            for (int i = 0; i < n; ++i) {
                cd t1 = Q[(size_t)i * n + k], t2 = Q[(size_t)i * n + k + 1];
                Q[(size_t)i * n + k] = cs * t1 + std::conj(sn) * t2;
                Q[(size_t)i * n + k + 1] = -sn * t1 + cs * t2;
            }
            if (k + 1 < hi) {
                x = A(k + 1, k);
                y = A(k + 2, k);
            }
        }
    }
    return 0;
}
}  // namespace

// Solve A X = B for X (A n x n, B n x r, row-major), Gaussian elimination with partial pivoting.
int dense_solve(int n, int r, std::vector<cd> A, std::vector<cd>& B) {
    for (int j = 0; j < n; ++j) {
        int p = j;
        for (int i = j + 1; i < n; ++i)
            if (std::abs(A[(size_t)i * n + j]) > std::abs(A[(size_t)p * n + j])) p = i;
        if (std::abs(A[(size_t)p * n + j]) == 0) return 1;
        if (p != j) {
            for (int l = 0; l < n; ++l) std::swap(A[(size_t)j * n + l], A[(size_t)p * n + l]);
            for (int l = 0; l < r; ++l) std::swap(B[(size_t)j * r + l], B[(size_t)p * r + l]);
        }
        for (int i = j + 1; i < n; ++i) {
            cd f = A[(size_t)i * n + j] / A[(size_t)j * n + j];
            if (f == 0.0) continue;
            for (int l = j; l < n; ++l) A[(size_t)i * n + l] -= f * A[(size_t)j * n + l];
            for (int l = 0; l < r; ++l) B[(size_t)i * r + l] -= f * B[(size_t)j * r + l];
        }
    }
    for (int i = n - 1; i >= 0; --i)
        for (int l = 0; l < r; ++l) {
            cd s = B[(size_t)i * r + l];
            for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * B[(size_t)j * r + l];
            B[(size_t)i * r + l] = s / A[(size_t)i * n + i];
        }
    return 0;
}

// Cholesky factor of a Hermitian positive definite G = R^dag R (R upper, row-major).
int cholesky_upper(int n, const std::vector<cd>& G, std::vector<cd>& Rf) {
    Rf.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double d = G[(size_t)i * n + i].real();
        for (int k = 0; k < i; ++k) d -= std::norm(Rf[(size_t)k * n + i]);
        if (!(d > 0)) return 1;
        double rii = std::sqrt(d);
        Rf[(size_t)i * n + i] = rii;
        for (int j = i + 1; j < n; ++j) {
            cd s = G[(size_t)i * n + j];
            for (int k = 0; k < i; ++k) s -= std::conj(Rf[(size_t)k * n + i]) * Rf[(size_t)k * n + j];
            Rf[(size_t)i * n + j] = s / rii;
        }
    }
    return 0;
}

}  // namespace sgn
