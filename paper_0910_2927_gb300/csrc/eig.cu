// Deflation set-up: the critical eigenpairs of A = H_W(mu) for LR deflation
// (Sec. 4, eq. (4.1)).  The paper takes R, L, Lambda as given; this file
// computes them on the GPU.
//
// Right eigenvectors: the m + extra eigenvalues of smallest |lambda|.  They are
// the eigenvalues of A^2 of smallest modulus, i.e. the low end of the
// spectrum of A^2, which a Chebyshev polynomial in A^2 amplifies.  For mu > 0
// A is not Hermitian and the eigenvalues of A^2 leave the real axis (|Im| of
// order 2 |lambda| |Im lambda|, about 1 at mu = 0.3), so the polynomial is the
// Chebyshev polynomial of an ellipse rather than of the interval [a, b]: real
// semi-axis (b - a)/2 from a (the top of the current block) to b (a bound of
// |lambda|^2), imaginary semi-axis beta from a short Arnoldi run on A^2.  On
// the interval alone the off-axis eigenvalues outgrow the wanted edge once the
// gap above it is small.  Block
// subspace iteration with that filter, SVQB orthonormalisation (Gram matrix,
// Hermitian eigendecomposition, rank-safe inverse square root) and
// Rayleigh-Ritz with A^2, where the wanted eigenvalues are extremal (with the
// indefinite A itself an unconverged block gives spurious Ritz values near 0,
// mixtures of eigenvectors of +lambda and -lambda).  Once the invariant
// subspace of A^2 has converged, one Rayleigh-Ritz step with A on it gives the
// eigenpairs of A, including pairs whose eigenvalues share a square.  The
// filter runs in FP32 until the residuals reach 1e-5, then in FP64.
// Left eigenvectors: the same on A^dag = H_W(-mu) (eigenvalues conj(lambda)).
// Finally L is rescaled to the dual basis, L <- L (L^dag R)^{-dag}, so that
// L^dag R = I.
#include "ctx.cuh"
#include "dense_eig.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>

namespace sgn {
namespace {

using cd = std::complex<double>;

template <class T>
cudaError_t hw(const sgn_ctx* c, T* out, const T* in, int ncol, bool adj, cudaStream_t st);
template <>
cudaError_t hw<double2>(const sgn_ctx* c, double2* out, const double2* in, int ncol, bool adj, cudaStream_t st) {
    return apply_hw64(c, out, in, ncol, adj, nullptr, st);
}
template <>
cudaError_t hw<float2>(const sgn_ctx* c, float2* out, const float2* in, int ncol, bool adj, cudaStream_t st) {
    return apply_hw32(c, out, in, ncol, adj, nullptr, st);
}

struct Work {
    sgn_ctx* c = nullptr;
    int q = 0;
    int64_t n = 0;
    DevBuf buf;
    void* blk[5] = {};  // Y, Yprev, Ynext, T1, T2 (q fields each, storage type of the phase)
    double2* partial = nullptr;
    int nblk = 0;
    int rstride = 0;
    DevState S{};
    double2* Cdev = nullptr;   // q x q coefficients
    double2* coef = nullptr;   // q x rstride per-column coefficients
    std::vector<double2> hred;
    double beta = 0;           // imaginary semi-axis of the filter ellipse
};

int setup(Work& W, sgn_ctx* c, int q, size_t esz, int nblk) {
    W.c = c;
    W.q = q;
    W.n = c->n;
    W.nblk = nblk;
    W.rstride = 104;
    const size_t blkb = (size_t)q * c->n * esz;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += (b + 255) & ~size_t(255);
        return o;
    };
    size_t ob[5];
    for (int i = 0; i < 5; ++i) ob[i] = take(blkb);
    size_t op = take((size_t)q * W.rstride * nblk * sizeof(double2));
    size_t ored = take((size_t)q * W.rstride * sizeof(double2));
    size_t oc = take((size_t)q * q * sizeof(double2));
    size_t ocoef = take((size_t)q * W.rstride * sizeof(double2));
    size_t oint = take((size_t)3 * q * sizeof(int));
    SGN_CHECK(dev_alloc(c, W.buf, off));
    char* b = reinterpret_cast<char*>(W.buf.p);
    for (int i = 0; i < 5; ++i) W.blk[i] = b + ob[i];
    W.partial = reinterpret_cast<double2*>(b + op);
    W.S.red = reinterpret_cast<double2*>(b + ored);
    W.Cdev = reinterpret_cast<double2*>(b + oc);
    W.coef = reinterpret_cast<double2*>(b + ocoef);
    W.S.skip = reinterpret_cast<int*>(b + oint);
    W.S.done = W.S.skip + q;
    W.S.kk = W.S.skip + 2 * q;
    W.S.rstride = W.rstride;
    SGN_CUDA(cudaMemsetAsync(W.buf.p, 0, off, c->work));
    W.hred.resize((size_t)q * W.rstride);
    return SGN_OK;
}

// G[i][j] = X_i^dag Y_j for p fields X and r fields Y (row-major p x r on the host).
template <class T>
int gram(Work& W, const T* X, int p, const T* Y, int r, std::vector<cd>& G) {
    cudaStream_t st = W.c->work;
    const Reduce rd{W.partial, W.nblk, W.rstride};
    SGN_CUDA(mdot<T>(Basis<T>{X, W.n, 0}, p, Y, W.n, W.n, r, rd, 0, nullptr, st));
    SGN_CUDA(reduce(rd, p, r, RM_STORE, 0, W.S, nullptr, st));
    SGN_CUDA(cudaMemcpyAsync(W.hred.data(), W.S.red, sizeof(double2) * r * W.rstride, cudaMemcpyDeviceToHost, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    G.assign((size_t)p * r, 0.0);
    for (int j = 0; j < r; ++j)
        for (int i = 0; i < p; ++i) {
            double2 v = W.hred[(size_t)j * W.rstride + i];
            G[(size_t)i * r + j] = cd(v.x, v.y);
        }
    return SGN_OK;
}

// Z = Y C (C host row-major q x r).
template <class T>
int combine(Work& W, const T* Y, int q, const std::vector<cd>& Cm, int r, T* Z) {
    cudaStream_t st = W.c->work;
    std::vector<double2> h((size_t)q * r);
    for (size_t i = 0; i < h.size(); ++i) h[i] = make_double2(Cm[i].real(), Cm[i].imag());
    SGN_CUDA(cudaMemcpyAsync(W.Cdev, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, st));
    SGN_CUDA(block_combine<T>(Y, q, W.Cdev, r, Z, W.n, st));
    SGN_CUDA(cudaStreamSynchronize(st));  // h is released on return
    return SGN_OK;
}

// Orthonormalise the q fields of Y in place (tmp: q fields of scratch).  SVQB:
// G = Y^dag Y, D = diag(G)^{-1/2}, D G D = V diag(l) V^dag, Y <- Y D V diag(l)^{-1/2}
// with l floored at eps * max(l) so that dependent columns do not blow up.
template <class T>
int svqb(Work& W, T* Y, int q, T* tmp, double eps, int* deficient = nullptr) {
    std::vector<cd> G;
    SGN_CHECK(gram<T>(W, Y, q, Y, q, G));
    std::vector<double> d(q);
    for (int i = 0; i < q; ++i) {
        double g = G[(size_t)i * q + i].real();
        d[i] = g > 0 ? 1.0 / std::sqrt(g) : 0.0;
    }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) G[(size_t)i * q + j] *= d[i] * d[j];
    for (int i = 0; i < q; ++i)  // make exactly Hermitian
        for (int j = 0; j < i; ++j) {
            cd a = 0.5 * (G[(size_t)i * q + j] + std::conj(G[(size_t)j * q + i]));
            G[(size_t)i * q + j] = a;
            G[(size_t)j * q + i] = std::conj(a);
        }
    std::vector<double> w;
    std::vector<cd> V;
    if (herm_eig(q, G, w, V)) {
        set_error("deflation set-up: eigendecomposition of the Gram matrix failed");
        return SGN_ERR_DEFLATION;
    }
    double lmax = 0;
    for (double l : w) lmax = std::max(lmax, l);
    std::vector<cd> Cm((size_t)q * q);
    std::vector<int> bad;
    for (int j = 0; j < q; ++j) {
        double l = w[j];
        if (!(l > eps * lmax)) {
            bad.push_back(j);
            l = lmax;  // the column is replaced below
        }
        double sc = 1.0 / std::sqrt(l);
        for (int i = 0; i < q; ++i) Cm[(size_t)i * q + j] = d[i] * V[(size_t)i * q + j] * sc;
    }
    SGN_CHECK(combine<T>(W, Y, q, Cm, q, tmp));
    SGN_CUDA(cudaMemcpyAsync(Y, tmp, sizeof(T) * q * W.n, cudaMemcpyDeviceToDevice, W.c->work));
    // numerically dependent directions carry no information: refill them with fresh
    // random fields, which the next orthonormalisation pass makes orthogonal
    static uint64_t refill_seed = 0x9a11ULL;
    for (int j : bad) SGN_CUDA(random_fill<T>(Y + (size_t)j * W.n, W.n, ++refill_seed, W.c->work));
    if (deficient) *deficient = (int)bad.size();
    return SGN_OK;
}

// Ellipse geometry of the filter: centre c0 = (a + b)/2, real semi-axis
// al = (b - a)/2, imaginary semi-axis beta < al, foci c0 -+ d, d = sqrt(al^2 - beta^2).
// The Chebyshev polynomial T_j((z - c0)/d) has modulus about r^j / 2 on the
// ellipse, r = (al + beta)/d, and grows as exp(j acosh((c0 - t)/d)) at a real t < a.
struct Ellipse {
    double c0, al, d, r;
    Ellipse(double a, double b, double beta) {
        c0 = 0.5 * (a + b);
        al = 0.5 * (b - a);
        d = std::sqrt(al * al - beta * beta);
        r = (al + beta) / d;
    }
    // growth exponent per degree at the real point t, relative to the ellipse
    double net(double t) const {
        const double x = (c0 - t) / d;
        return (x > 1.0 ? std::acosh(x) : 0.0) - std::log(r);
    }
};

// Chebyshev filter T_deg((A^2 - c0)/d) Y / r^deg, in place: the scaled
// recurrence y_{j+1} = (2/r) s y_j - y_{j-1}/r^2, s = (A^2 - c0)/d, keeps the
// components on the ellipse at O(1) and the wanted ones below the cap `amp`.
template <class T>
int filter(Work& W, bool adj, T* Y, double a, double b, int deg) {
    cudaStream_t st = W.c->work;
    const int q = W.q;
    const int64_t cnt = (int64_t)q * W.n;
    T* Yp = reinterpret_cast<T*>(W.blk[1]);
    T* Yn = reinterpret_cast<T*>(W.blk[2]);
    T* T1 = reinterpret_cast<T*>(W.blk[3]);
    T* T2 = reinterpret_cast<T*>(W.blk[4]);
    const Ellipse e(a, b, W.beta);
    const double al = 1.0 / (e.d * e.r), be = -e.c0 / (e.d * e.r);
    T* cur = Y;
    // Y1 = s(A^2) Y0 / r
    SGN_CUDA(hw<T>(W.c, T1, cur, q, adj, st));
    SGN_CUDA(hw<T>(W.c, T2, T1, q, adj, st));
    SGN_CUDA(cudaMemcpyAsync(Yp, cur, sizeof(T) * cnt, cudaMemcpyDeviceToDevice, st));
    SGN_CUDA(axpby3<T>(Yn, al, T2, be, Yp, 0.0, nullptr, cnt, st));
    T* prev = Yp;
    T* now = Yn;
    T* spare = cur;
    const double rr2 = 1.0 / (e.r * e.r);
    for (int j = 1; j < deg; ++j) {
        SGN_CUDA(hw<T>(W.c, T1, now, q, adj, st));
        SGN_CUDA(hw<T>(W.c, T2, T1, q, adj, st));
        SGN_CUDA(axpby3<T>(spare, 2 * al, T2, 2 * be, now, -rr2, prev, cnt, st));
        T* t = prev;
        prev = now;
        now = spare;
        spare = t;
    }
    if (now != Y) SGN_CUDA(cudaMemcpyAsync(Y, now, sizeof(T) * cnt, cudaMemcpyDeviceToDevice, st));
    return SGN_OK;
}

// Largest |Im theta| over the Ritz values of K Arnoldi steps on A^2 (CGS2,
// one random start field): an estimate of the imaginary extent of the
// spectrum of A^2, whose outer boundary Arnoldi resolves first.  Scratch:
// blocks 1 (the K + 1 basis fields), 3 and 4.
template <class T>
int spectrum_height2(Work& W, bool adj, int K, uint64_t seed, double* height) {
    cudaStream_t st = W.c->work;
    const int64_t n = W.n;
    K = std::min(K, W.q - 1);
    T* V = reinterpret_cast<T*>(W.blk[1]);
    T* w = reinterpret_cast<T*>(W.blk[3]);
    T* t = reinterpret_cast<T*>(W.blk[4]);
    std::vector<cd> Hh((size_t)K * K, 0.0), G;
    SGN_CUDA(random_fill<T>(V, n, seed, st));
    SGN_CHECK(gram<T>(W, V, 1, V, 1, G));
    SGN_CUDA(axpby3<T>(V, 1.0 / std::sqrt(G[0].real()), V, 0.0, V, 0.0, nullptr, n, st));
    int k = K;
    for (int j = 0; j < K; ++j) {
        T* vj = V + (size_t)j * n;
        T* vn = V + (size_t)(j + 1) * n;
        SGN_CUDA(hw<T>(W.c, t, vj, 1, adj, st));
        SGN_CUDA(hw<T>(W.c, w, t, 1, adj, st));
        // two classical Gram-Schmidt passes against v_0..v_j
        std::vector<cd> h;
        SGN_CHECK(gram<T>(W, V, j + 1, w, 1, h));
        SGN_CHECK(combine<T>(W, V, j + 1, h, 1, t));
        SGN_CUDA(axpby3<T>(vn, 1.0, w, -1.0, t, 0.0, nullptr, n, st));
        std::vector<cd> h2;
        SGN_CHECK(gram<T>(W, V, j + 1, vn, 1, h2));
        SGN_CHECK(combine<T>(W, V, j + 1, h2, 1, t));
        SGN_CUDA(axpby3<T>(w, 1.0, vn, -1.0, t, 0.0, nullptr, n, st));
        for (int i = 0; i <= j; ++i) Hh[(size_t)i * K + j] = h[i] + h2[i];
        SGN_CHECK(gram<T>(W, w, 1, w, 1, G));
        const double nrm = std::sqrt(std::max(G[0].real(), 0.0));
        double hn = 0;
        for (int i = 0; i <= j; ++i) hn += std::norm(Hh[(size_t)i * K + j]);
        if (!(nrm > 1e-10 * std::sqrt(hn))) {  // invariant subspace: the Ritz values are exact
            k = j + 1;
            break;
        }
        if (j + 1 < K) Hh[(size_t)(j + 1) * K + j] = nrm;
        SGN_CUDA(axpby3<T>(vn, 1.0 / nrm, w, 0.0, w, 0.0, nullptr, n, st));
    }
    std::vector<cd> Hk((size_t)k * k);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Hk[(size_t)i * k + j] = Hh[(size_t)i * K + j];
    std::vector<cd> th, X;
    if (dense_eig(k, Hk, th, X)) {
        set_error("deflation set-up: Arnoldi eigendecomposition failed");
        return SGN_ERR_DEFLATION;
    }
    double hmax = 0;
    for (const cd& z : th) hmax = std::max(hmax, std::abs(z.imag()));
    *height = hmax;
    return SGN_OK;
}

struct Ritz {
    std::vector<cd> theta;
    std::vector<double> res;  // relative eigen-residuals
};

bool ritz_less(cd a, cd b) {
    if (std::abs(a) != std::abs(b)) return std::abs(a) < std::abs(b);
    if (a.real() != b.real()) return a.real() < b.real();
    return a.imag() < b.imag();
}

// Rayleigh-Ritz with M = A^2 (squared) or M = A on span(Y), Y orthonormal (q
// fields): Y <- normalised Ritz vectors sorted by |theta|, with their relative
// eigen-residuals ||M y - theta y|| / |theta|.
template <class T>
int rayleigh_ritz(Work& W, bool adj, bool squared, T* Y, int q, Ritz& out) {
    cudaStream_t st = W.c->work;
    T* Z = reinterpret_cast<T*>(W.blk[3]);
    T* Yw = reinterpret_cast<T*>(W.blk[1]);
    T* Zw = reinterpret_cast<T*>(W.blk[2]);
    if (squared) {
        T* T1 = reinterpret_cast<T*>(W.blk[4]);
        SGN_CUDA(hw<T>(W.c, T1, Y, q, adj, st));
        SGN_CUDA(hw<T>(W.c, Z, T1, q, adj, st));
    } else {
        SGN_CUDA(hw<T>(W.c, Z, Y, q, adj, st));
    }
    std::vector<cd> G;
    SGN_CHECK(gram<T>(W, Y, q, Z, q, G));
    std::vector<cd> w, X;
    if (dense_eig(q, G, w, X)) {
        set_error("deflation set-up: Rayleigh-Ritz eigendecomposition failed");
        return SGN_ERR_DEFLATION;
    }
    std::vector<int> ord(q);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int i, int j) { return ritz_less(w[i], w[j]); });
    std::vector<cd> Xs((size_t)q * q);
    out.theta.resize(q);
    for (int j = 0; j < q; ++j) {
        out.theta[j] = w[ord[j]];
        for (int i = 0; i < q; ++i) Xs[(size_t)i * q + j] = X[(size_t)i * q + ord[j]];
    }
    SGN_CHECK(combine<T>(W, Y, q, Xs, q, Yw));
    SGN_CHECK(combine<T>(W, Z, q, Xs, q, Zw));
    // residuals ||Z_j - theta_j Y_j||, ||Y_j||
    std::vector<double2> th((size_t)q * W.rstride, make_double2(0, 0));
    for (int j = 0; j < q; ++j) th[(size_t)j * W.rstride] = make_double2(out.theta[j].real(), out.theta[j].imag());
    SGN_CUDA(cudaMemcpyAsync(W.coef, th.data(), sizeof(double2) * th.size(), cudaMemcpyHostToDevice, st));
    const Reduce rd{W.partial, W.nblk, W.rstride};
    SGN_CUDA(mdot<T>(Basis<T>{Yw, 0, W.n}, 0, Yw, W.n, W.n, q, rd, 1, nullptr, st));
    SGN_CUDA(reduce(rd, 1, q, RM_STORE, 0, W.S, nullptr, st));
    SGN_CUDA(cudaMemcpyAsync(W.hred.data(), W.S.red, sizeof(double2) * q * W.rstride, cudaMemcpyDeviceToHost, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    std::vector<double> ynorm(q);
    for (int j = 0; j < q; ++j) ynorm[j] = std::sqrt(W.hred[(size_t)j * W.rstride].x);
    SGN_CUDA(maxpy_mdot<T>(Basis<T>{Yw, 0, W.n}, 1, W.coef, W.rstride, Zw, W.n, W.n, q, rd, nullptr, st));
    SGN_CUDA(reduce(rd, 2, q, RM_STORE, 0, W.S, nullptr, st));
    SGN_CUDA(cudaMemcpyAsync(W.hred.data(), W.S.red, sizeof(double2) * q * W.rstride, cudaMemcpyDeviceToHost, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    out.res.resize(q);
    for (int j = 0; j < q; ++j) {
        double rn = std::sqrt(std::max(W.hred[(size_t)j * W.rstride + 1].x, 0.0));
        double den = std::abs(out.theta[j]) * (ynorm[j] > 0 ? ynorm[j] : 1.0);
        out.res[j] = den > 0 ? rn / den : INFINITY;
    }
    // Y <- normalised Ritz vectors
    std::vector<double> sc(q);
    for (int j = 0; j < q; ++j) sc[j] = ynorm[j] > 0 ? 1.0 / ynorm[j] : 0.0;
    std::vector<cd> Dm((size_t)q * q, 0.0);
    for (int j = 0; j < q; ++j) Dm[(size_t)j * q + j] = sc[j];
    SGN_CHECK(combine<T>(W, Yw, q, Dm, q, Y));
    return SGN_OK;
}

// Upper bound of |lambda|^2 over the spectrum of A: with the orthogonal spin
// projectors (1 -/+ gamma)/2, each hop pair of direction nu has norm at most
// sqrt(e^{2 mu d} + e^{-2 mu d}), so ||A|| <= |4 + m_W| + 3 sqrt(2) + sqrt(2 cosh 2mu).
double spectral_bound2(const sgn_ctx* c) {
    double nb = std::abs(4.0 + c->mass) + 3.0 * std::sqrt(2.0) + std::sqrt(2.0 * std::cosh(2.0 * c->mu));
    return nb * nb * 1.0001;
}

int degree_for(const Ellipse& e, double t, double amp, int dmax) {
    const double g = e.net(t);
    if (!(g > 1e-12)) return dmax;
    const int di = (int)std::ceil(std::acosh(amp) / g);
    return std::min(dmax, std::max(4, di));
}

bool debug_on() {
    static const bool on = [] {
        const char* s = getenv("SGN_DEBUG");
        return s && s[0] == '1';
    }();
    return on;
}

// Iterate until the wanted Ritz pairs of A^2 reach `tol`, or (stop_on_stall)
// until the worst residual stops improving: the FP32 phase cannot go below
// its rounding floor, about eps_32 ||A^2|| / |theta|.
template <class T>
int iterate(Work& W, bool adj, T* Y, int want, double tol, int max_it, Ritz& rz, bool fresh, bool stop_on_stall,
            int* its) {
    const int q = W.q;
    const double b = spectral_bound2(W.c);
    T* tmp = reinterpret_cast<T*>(W.blk[1]);
    const bool f64 = sizeof(T) == 16;
    // Gram eigenvalues below eps * max are unresolved (FP64 Gram of FP64 data to
    // ~1e-16; of FP32 data, with FP32 chunk products, to ~1e-7)
    const double eps = f64 ? 1e-14 : 1e-7;
    if (fresh) {
        SGN_CHECK(svqb<T>(W, Y, q, tmp, eps));
        SGN_CHECK(svqb<T>(W, Y, q, tmp, eps));
        SGN_CHECK(rayleigh_ritz<T>(W, adj, true, Y, q, rz));
    }
    double best = INFINITY;
    int stall = 0;
    for (int it = 0; it < max_it; ++it) {
        double worst = 0;
        for (int j = 0; j < want; ++j) worst = std::max(worst, rz.res[j]);
        if (debug_on())
            fprintf(stderr,
                    "[sgn eig %s %s] it %d worst %.3e theta_min %.4e theta_want %.4e theta_top %.4e beta %.3f\n",
                    adj ? "left" : "right", f64 ? "fp64" : "fp32", it, worst, std::abs(rz.theta[0]),
                    std::abs(rz.theta[want - 1]), std::abs(rz.theta[q - 1]), W.beta);
        if (worst <= tol) {
            *its = it;
            return SGN_OK;
        }
        if (stop_on_stall) {
            if (worst < 0.5 * best) {
                best = worst;
                stall = 0;
            } else if (++stall >= 2) {
                *its = it;
                return SGN_OK;
            }
        }
        // Ritz values are eigenvalue estimates of A^2: |theta| ~ |lambda|^2.  The
        // degree aims at an amplification of the wanted edge tw, capped so that the
        // most amplified direction (the smallest Ritz value) outgrows the top of the
        // block by less than the storage precision can resolve.
        const double tw = std::abs(rz.theta[want - 1]);
        const double tmin = std::abs(rz.theta[0]);
        double a = std::abs(rz.theta[q - 1]);
        a = std::max(a, 1.02 * tw);
        a = std::min(a, std::min(0.9 * b, b - 4.0 * W.beta));  // keeps beta below half the real semi-axis
        const int dmax = f64 ? 400 : 800;
        const double amp = f64 ? 1e6 : 1e3;  // squared stays inside the Gram resolution above
        const Ellipse e(a, b, W.beta);
        const int d_conv = degree_for(e, tw, amp, dmax);
        const int d_safe = degree_for(e, tmin, amp, dmax);
        const int deg = std::max(4, std::min(d_conv, d_safe));
        SGN_CHECK(filter<T>(W, adj, Y, a, b, deg));
        int bad = 0;
        SGN_CHECK(svqb<T>(W, Y, q, tmp, eps, &bad));
        SGN_CHECK(svqb<T>(W, Y, q, tmp, eps));
        if (bad) SGN_CHECK(svqb<T>(W, Y, q, tmp, eps));
        if (debug_on() && bad) fprintf(stderr, "[sgn eig] refilled %d dependent directions\n", bad);
        SGN_CHECK(rayleigh_ritz<T>(W, adj, true, Y, q, rz));
    }
    double worst = 0;
    for (int j = 0; j < want; ++j) worst = std::max(worst, rz.res[j]);
    *its = max_it;
    if (worst <= tol || stop_on_stall) return SGN_OK;
    char msg[160];
    snprintf(msg, sizeof msg, "deflation set-up: eigenpairs did not converge in %d iterations (worst relative residual %.3e, tolerance %.3e)",
             max_it, worst, tol);
    set_error(msg);
    return SGN_ERR_DEFLATION;
}

// Orthonormalise the `want` fields F (block 4) and run Rayleigh-Ritz with A on
// them; the eigenvector estimates replace F.  Scratch: blocks 1..3.
int svqb_final(Work& W, double2* F, int want, bool adj, Ritz& ra) {
    double2* tmp = reinterpret_cast<double2*>(W.blk[1]);
    SGN_CHECK(svqb<double2>(W, F, want, tmp, 1e-15));
    SGN_CHECK(svqb<double2>(W, F, want, tmp, 1e-15));
    return rayleigh_ritz<double2>(W, adj, false, F, want, ra);
}

// One side: `want` eigenpairs of A (adj = false) or A^dag (adj = true) into V64 (want fields, FP64).
int eig_side(sgn_ctx* c, bool adj, int want, int q, double tol, uint64_t seed, double2* V64, std::vector<cd>& lam) {
    cudaStream_t st = c->work;
    Ritz rz;
    int its = 0;
    Work W;
    SGN_CHECK(setup(W, c, q, sizeof(float2), reduce_blocks<float2>(c->n)));
    float2* Y = reinterpret_cast<float2*>(W.blk[0]);
    // imaginary extent of the spectrum of A^2, widened by 15 % (Arnoldi Ritz
    // values approach the outer boundary of the spectrum from inside)
    double height = 0;
    int rc = spectrum_height2<float2>(W, adj, 40, seed ^ 0xa5a5ULL, &height);
    if (rc != SGN_OK) {
        dev_free(c, W.buf);
        return rc;
    }
    W.beta = 1.15 * height;
    if (debug_on()) fprintf(stderr, "[sgn eig] spectrum of A^2: max |Im| %.4f (Arnoldi)\n", height);
    SGN_CUDA(random_fill<float2>(Y, (int64_t)q * c->n, seed, st));
    // FP32 filter until the A^2 residuals reach their FP32 floor (or tol)
    rc = iterate<float2>(W, adj, Y, want, std::max(tol, 1e-6), 80, rz, true, true, &its);
    if (rc != SGN_OK) {
        dev_free(c, W.buf);
        return rc;
    }
    Work W64;
    rc = setup(W64, c, q, sizeof(double2), reduce_blocks<double2>(c->n));
    if (rc != SGN_OK) {
        dev_free(c, W.buf);
        return rc;
    }
    W64.beta = W.beta;
    double2* Y64 = reinterpret_cast<double2*>(W64.blk[0]);
    SGN_CUDA(convert_f32_to_f64(Y, Y64, (int64_t)q * c->n, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    dev_free(c, W.buf);
    // FP64: converge the A^2 subspace, then split it with one Rayleigh-Ritz step on A
    double tol2 = tol / 10;
    for (int attempt = 0; attempt < 4 && rc == SGN_OK; ++attempt) {
        rc = iterate<double2>(W64, adj, Y64, want, tol2, 40, rz, attempt == 0, false, &its);
        if (rc != SGN_OK) break;
        double2* F = reinterpret_cast<double2*>(W64.blk[4]);
        SGN_CUDA(cudaMemcpyAsync(F, Y64, sizeof(double2) * want * c->n, cudaMemcpyDeviceToDevice, st));
        Ritz ra;
        rc = svqb_final(W64, F, want, adj, ra);
        if (rc != SGN_OK) break;
        double worst = 0;
        for (int j = 0; j < want; ++j) worst = std::max(worst, ra.res[j]);
        if (worst <= tol) {
            SGN_CUDA(cudaMemcpyAsync(V64, F, sizeof(double2) * want * c->n, cudaMemcpyDeviceToDevice, st));
            SGN_CUDA(cudaStreamSynchronize(st));
            lam = ra.theta;
            dev_free(c, W64.buf);
            return SGN_OK;
        }
        tol2 /= 10;
    }
    dev_free(c, W64.buf);
    if (rc == SGN_OK) {
        set_error("deflation set-up: eigenpairs of A did not reach the tolerance");
        rc = SGN_ERR_DEFLATION;
    }
    return rc;
}

}  // namespace

int build_deflation(sgn_ctx* c, int m, int extra, double eig_tol, double* lambda_out) {
    cudaStream_t st = c->work;
    const int want = m + extra;
    const int q = std::min(100, want + std::max(12, want / 2));
    const int64_t n = c->n;
    DevBuf RL;
    SGN_CHECK(dev_alloc(c, RL, sizeof(double2) * (size_t)n * (3 * want)));
    double2* Rw = reinterpret_cast<double2*>(RL.p);
    double2* Lw = Rw + (size_t)want * n;
    double2* Lm = Lw + (size_t)want * n;
    std::vector<cd> lamR, lamL;
    int rc = eig_side(c, false, want, q, eig_tol, 0x5eed0001ULL, Rw, lamR);
    if (rc == SGN_OK) rc = eig_side(c, true, want, q, eig_tol, 0x5eed0002ULL, Lw, lamL);
    if (rc != SGN_OK) {
        dev_free(c, RL);
        return rc;
    }
    // the selection must be unambiguous: |lambda_m| < |lambda_{m+1}|
    if (extra > 0 && !(std::abs(lamR[m]) - std::abs(lamR[m - 1]) > 1e-8 * std::abs(lamR[m - 1]))) {
        dev_free(c, RL);
        set_error("deflation set-up: |lambda_m| and |lambda_m+1| coincide; choose another m");
        return SGN_ERR_DEFLATION;
    }
    // pair every right eigenvalue with the left one whose conjugate is closest (all
    // `want` pairs: the m deflated ones and the extra ones kept for the derivative)
    std::vector<int> pick(want, -1);
    std::vector<char> used(want, 0);
    for (int j = 0; j < want; ++j) {
        double best = INFINITY;
        for (int l = 0; l < want; ++l) {
            if (used[l]) continue;
            double d = std::abs(lamR[j] - std::conj(lamL[l]));
            if (d < best) {
                best = d;
                pick[j] = l;
            }
        }
        used[pick[j]] = 1;
        if (best > 1e-6 * std::max(1.0, std::abs(lamR[j]))) {
            dev_free(c, RL);
            set_error("deflation set-up: left and right spectra do not match");
            return SGN_ERR_DEFLATION;
        }
    }
    for (int j = 0; j < want; ++j)
        SGN_CUDA(cudaMemcpyAsync(Lm + (size_t)j * n, Lw + (size_t)pick[j] * n, sizeof(double2) * n,
                                 cudaMemcpyDeviceToDevice, st));
    // L <- L M^{-dag}, M = L^dag R  (then L^dag R = I over all want pairs)
    const int w2 = want;
    {
        Work W;
        rc = setup(W, c, w2, sizeof(double2), reduce_blocks<double2>(n));
        std::vector<cd> M;
        if (rc == SGN_OK) rc = gram<double2>(W, Lm, w2, Rw, w2, M);
        std::vector<cd> Mh((size_t)w2 * w2), X((size_t)w2 * w2, 0.0);
        if (rc == SGN_OK) {
            for (int i = 0; i < w2; ++i)
                for (int j = 0; j < w2; ++j) Mh[(size_t)i * w2 + j] = std::conj(M[(size_t)j * w2 + i]);
            for (int i = 0; i < w2; ++i) X[(size_t)i * w2 + i] = 1.0;
            if (dense_solve(w2, w2, Mh, X)) {
                set_error("deflation set-up: L^dag R is singular");
                rc = SGN_ERR_DEFLATION;
            }
        }
        // X = M^{-dag}; L_new = L X, written to the Lw slot
        if (rc == SGN_OK) rc = combine<double2>(W, Lm, w2, X, w2, Lw);
        std::vector<cd> chk;
        if (rc == SGN_OK) rc = gram<double2>(W, Lw, w2, Rw, w2, chk);
        if (rc == SGN_OK) {
            double e = 0;
            for (int i = 0; i < w2; ++i)
                for (int j = 0; j < w2; ++j) e = std::max(e, std::abs(chk[(size_t)i * w2 + j] - (i == j ? 1.0 : 0.0)));
            if (!(e < 1e-8)) {
                set_error("deflation set-up: biorthonormalisation failed (||L^dag R - I|| = " + std::to_string(e) +
                          ")");
                rc = SGN_ERR_DEFLATION;
            }
        }
        dev_free(c, W.buf);
        if (rc != SGN_OK) {
            dev_free(c, RL);
            return rc;
        }
    }
    // install as the context's deflation data
    const size_t cnt = (size_t)n * m;
    SGN_CHECK(dev_alloc(c, c->R64, cnt * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->L64, cnt * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->R32, cnt * sizeof(float2)));
    SGN_CHECK(dev_alloc(c, c->L32, cnt * sizeof(float2)));
    SGN_CHECK(dev_alloc(c, c->lam_dev, (size_t)m * sizeof(double2)));
    SGN_CHECK(dev_alloc(c, c->lamc_dev, (size_t)m * sizeof(double2)));
    SGN_CUDA(cudaMemcpyAsync(c->R64.p, Rw, cnt * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SGN_CUDA(cudaMemcpyAsync(c->L64.p, Lw, cnt * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SGN_CUDA(convert_f64_to_f32(as<double2>(c->R64), as<float2>(c->R32), (int64_t)cnt, st));
    SGN_CUDA(convert_f64_to_f32(as<double2>(c->L64), as<float2>(c->L32), (int64_t)cnt, st));
    std::vector<double2> hl(m), hlc(m);
    for (int j = 0; j < m; ++j) {
        hl[j] = make_double2(lamR[j].real(), lamR[j].imag());
        hlc[j] = make_double2(lamR[j].real(), -lamR[j].imag());
    }
    SGN_CUDA(cudaMemcpyAsync(c->lam_dev.p, hl.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, st));
    SGN_CUDA(cudaMemcpyAsync(c->lamc_dev.p, hlc.data(), sizeof(double2) * m, cudaMemcpyHostToDevice, st));
    // the extra pairs, for the derivative's reduced resolvents
    const int mx = want - m;
    if (mx > 0) {
        const size_t cx = (size_t)n * mx;
        SGN_CHECK(dev_alloc(c, c->Rx64, cx * sizeof(double2)));
        SGN_CHECK(dev_alloc(c, c->Lx64, cx * sizeof(double2)));
        SGN_CUDA(cudaMemcpyAsync(c->Rx64.p, Rw + (size_t)m * n, cx * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        SGN_CUDA(cudaMemcpyAsync(c->Lx64.p, Lw + (size_t)m * n, cx * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    SGN_CUDA(cudaStreamSynchronize(st));
    dev_free(c, RL);
    c->lam.assign(lamR.begin(), lamR.begin() + m);
    c->m = m;
    c->mx = mx;
    c->lamx.assign(lamR.begin() + m, lamR.begin() + want);
    if (lambda_out)
        for (int j = 0; j < want; ++j) {
            lambda_out[2 * j] = lamR[j].real();
            lambda_out[2 * j + 1] = lamR[j].imag();
        }
    return SGN_OK;
}

}  // namespace sgn
