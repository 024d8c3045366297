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
// The FP32 phase always reads the FP32 links: with BF16 or FP16 ones (a choice for the solves)
// its residuals would stall at the links' rounding instead of near the FP32 floor.
template <>
cudaError_t hw<float2>(const sgn_ctx* c, float2* out, const float2* in, int ncol, bool adj, cudaStream_t st) {
    return apply_hw32(c, out, in, ncol, adj, nullptr, st, true);
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
    // the polynomial filter is too weak for this spectrum (the ellipse enclosing the
    // unwanted eigenvalues of A^2 comes too close to the wanted ones): set by iterate()
    bool weak = false;
    DevBuf backup;  // copy of the block before a filter pass (allocated on first use)
    Work() = default;
    Work(const Work&) = delete;
    Work& operator=(const Work&) = delete;
    ~Work() {  // dev_free ignores buffers already released
        if (c) {
            dev_free(c, buf);
            dev_free(c, backup);
        }
    }
};

int setup(Work& W, sgn_ctx* c, int q, size_t esz, int nblk, int nblocks = 5) {
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
    size_t ob[5] = {};
    for (int i = 0; i < nblocks; ++i) ob[i] = take(blkb);
    size_t op = take((size_t)q * W.rstride * nblk * sizeof(double2));
    size_t ored = take((size_t)q * W.rstride * sizeof(double2));
    size_t oc = take((size_t)q * q * sizeof(double2));
    size_t ocoef = take((size_t)q * W.rstride * sizeof(double2));
    size_t oint = take((size_t)3 * q * sizeof(int));
    SGN_CHECK(dev_alloc(c, W.buf, off));
    char* b = reinterpret_cast<char*>(W.buf.p);
    for (int i = 0; i < 5; ++i) W.blk[i] = i < nblocks ? b + ob[i] : nullptr;
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
int svqb(Work& W, T* Y, int q, T* tmp, double eps, int* deficient = nullptr, bool* overflow = nullptr) {
    std::vector<cd> G;
    SGN_CHECK(gram<T>(W, Y, q, Y, q, G));
    if (overflow) {  // a filtered block that left the representable range: Y untouched
        *overflow = false;
        for (int i = 0; i < q; ++i) {
            const double g = G[(size_t)i * q + i].real();
            if (!std::isfinite(g)) *overflow = true;
        }
        if (*overflow) return SGN_OK;
    }
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
// spectrum of A^2, whose outer boundary Arnoldi resolves first.  The estimate
// falls short on large lattices when K is small (40 steps: 0.135 against a true
// height near 0.9 at 24^4, mu = 0.2; 200 steps recover most of it), and an
// ellipse that is too flat lets bulk eigenvalues outgrow the wanted ones, so K
// is 200 (or n - 1).  The basis lives in its own allocation (K + 1 fields of T);
// Gram-Schmidt runs in chunks of at most 96 basis vectors (the reduction's slots).
template <class T>
int spectrum_height2(Work& W, bool adj, int K, uint64_t seed, double* height) {
    cudaStream_t st = W.c->work;
    const int64_t n = W.n;
    K = (int)std::min<int64_t>(K, n - 1);
    DevBuf vb;
    SGN_CHECK(dev_alloc(W.c, vb, sizeof(T) * (size_t)(K + 1) * n));
    T* V = reinterpret_cast<T*>(vb.p);
    T* w = reinterpret_cast<T*>(W.blk[3]);
    T* t = reinterpret_cast<T*>(W.blk[4]);
    constexpr int CH = 96;
    std::vector<cd> Hh((size_t)K * K, 0.0), G;
    int k = K;
    auto body = [&]() -> int {
        SGN_CUDA(random_fill<T>(V, n, seed, st));
        SGN_CHECK(gram<T>(W, V, 1, V, 1, G));
        SGN_CUDA(axpby3<T>(V, 1.0 / std::sqrt(G[0].real()), V, 0.0, V, 0.0, nullptr, n, st));
        for (int j = 0; j < K; ++j) {
            T* vj = V + (size_t)j * n;
            T* vn = V + (size_t)(j + 1) * n;
            SGN_CUDA(hw<T>(W.c, t, vj, 1, adj, st));
            SGN_CUDA(hw<T>(W.c, w, t, 1, adj, st));
            // two classical Gram-Schmidt passes against v_0..v_j: all coefficients of a pass
            // from the same vector, subtracted chunk by chunk
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<cd> h(j + 1), hc;
                for (int c0 = 0; c0 <= j; c0 += CH) {
                    const int nc = std::min(CH, j + 1 - c0);
                    SGN_CHECK(gram<T>(W, V + (size_t)c0 * n, nc, w, 1, hc));
                    for (int i = 0; i < nc; ++i) h[c0 + i] = hc[i];
                }
                for (int c0 = 0; c0 <= j; c0 += CH) {
                    const int nc = std::min(CH, j + 1 - c0);
                    std::vector<cd> hs(h.begin() + c0, h.begin() + c0 + nc);
                    SGN_CHECK(combine<T>(W, V + (size_t)c0 * n, nc, hs, 1, t));
                    SGN_CUDA(axpby3<T>(w, 1.0, w, -1.0, t, 0.0, nullptr, n, st));
                }
                for (int i = 0; i <= j; ++i) Hh[(size_t)i * K + j] += h[i];
            }
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
        return SGN_OK;
    };
    const int rc = body();
    SGN_CUDA(cudaStreamSynchronize(st));
    dev_free(W.c, vb);
    SGN_CHECK(rc);
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
        // the first passes move the block from the middle of the spectrum to its low end and
        // do not count towards a stall
        if (worst < 0.5 * best || it < 3) {
            best = std::min(best, worst);
            stall = 0;
        } else if (++stall >= (stop_on_stall ? 2 : 8)) {
            *its = it;
            if (stop_on_stall) return SGN_OK;
            W.weak = true;
            set_error("deflation set-up: the polynomial filter stalled");
            return SGN_ERR_DEFLATION;
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
        // on the first pass of a fresh random block the cap also holds at t = 0: its Ritz
        // values sit in the middle of the spectrum, far above the smallest eigenvalues, which
        // a degree sized on them would amplify past the FP32 range
        const double tlow = (fresh && it == 0) ? std::min(tmin, 0.0) : tmin;
        const int d_conv = degree_for(e, tw, amp, dmax);
        const int d_safe = degree_for(e, tlow, amp, dmax);
        const int deg = std::max(4, std::min(d_conv, d_safe));
        // keep the block: a filter on too flat an ellipse amplifies bulk eigenvalues outside
        // it without bound, until the FP32 block overflows; then the pass is repeated with a
        // taller ellipse (by a quarter) and half the degree
        if (!W.backup.p) SGN_CHECK(dev_alloc(W.c, W.backup, sizeof(T) * (size_t)q * W.n));
        SGN_CUDA(cudaMemcpyAsync(W.backup.p, Y, sizeof(T) * (size_t)q * W.n, cudaMemcpyDeviceToDevice, W.c->work));
        int bad = 0;
        bool over = false;
        int dpass = deg;
        for (int tries = 0;; ++tries) {
            SGN_CHECK(filter<T>(W, adj, Y, a, b, dpass));
            SGN_CHECK(svqb<T>(W, Y, q, tmp, eps, &bad, &over));
            if (!over) break;
            if (tries >= 6 || !(4.0 * W.beta * 1.25 < b - a)) {
                set_error("deflation set-up: the filtered block overflows (spectrum outside the filter ellipse)");
                return SGN_ERR_DEFLATION;
            }
            W.beta *= 1.25;
            dpass = std::max(4, dpass / 2);
            if (debug_on())
                fprintf(stderr, "[sgn eig] filtered block overflowed: ellipse height -> %.3f, degree %d\n", W.beta,
                        dpass);
            SGN_CUDA(cudaMemcpyAsync(Y, W.backup.p, sizeof(T) * (size_t)q * W.n, cudaMemcpyDeviceToDevice,
                                     W.c->work));
        }
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

// ---- shift-invert Arnoldi ------------------------------------------------------
// Where the unwanted eigenvalues of A^2 nearly surround the wanted ones (strongly
// non-Hermitian A: at mu = 1 they lie on three sides of the disc |z| < |lambda_m+1|^2),
// no polynomial in A^2 separates them: the filter stalls, and a Krylov solver for
// A^2 (restarted GMRES) stagnates for the same reason.  The eigenvalues of smallest
// modulus of A are the largest of A^{-1}, well separated from the rest: Arnoldi on
// A^{-1} with thick restarts (the Ritz vectors of the wanted values are kept, a
// Krylov decomposition in Stewart's sense), every A^{-1} v by CGLS -- conjugate
// gradients on the normal equations A^dag A x = A^dag v, which converge for any
// eigenvalue distribution at a rate set by sigma_max / sigma_min of A.

struct CglsVecs {
    double2 *x, *r, *s, *p, *q;  // r and s adjacent (one Gram call gives both norms)
};

// x = A^{-1} b (A^dag with adj) until ||b - A x|| <= tol ||b|| or max_it steps.
int cgls(Work& W, bool adj, const double2* b, const CglsVecs& v, double tol, int max_it, int* its, double* relres) {
    sgn_ctx* c = W.c;
    cudaStream_t st = c->work;
    const int64_t n = W.n;
    std::vector<cd> G;
    SGN_CHECK(gram<double2>(W, b, 1, b, 1, G));
    const double bn = std::sqrt(std::max(G[0].real(), 0.0));
    SGN_CUDA(cudaMemsetAsync(v.x, 0, sizeof(double2) * n, st));
    *its = 0;
    *relres = 0;
    if (!(bn > 0)) return SGN_OK;
    SGN_CUDA(cudaMemcpyAsync(v.r, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    SGN_CUDA(apply_hw64(c, v.s, v.r, 1, !adj, nullptr, st));  // s = A^dag r (H_W(mu)^dag = H_W(-mu))
    SGN_CUDA(cudaMemcpyAsync(v.p, v.s, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    SGN_CHECK(gram<double2>(W, v.s, 1, v.s, 1, G));
    double gamma = G[0].real();
    double rn = bn;
    int it = 0;
    while (it < max_it) {
        SGN_CUDA(apply_hw64(c, v.q, v.p, 1, adj, nullptr, st));  // q = A p
        SGN_CHECK(gram<double2>(W, v.q, 1, v.q, 1, G));
        const double delta = G[0].real();
        if (!(delta > 0) || !std::isfinite(delta)) break;
        const double alpha = gamma / delta;
        SGN_CUDA(axpby3<double2>(v.x, 1.0, v.x, alpha, v.p, 0.0, nullptr, n, st));
        SGN_CUDA(axpby3<double2>(v.r, 1.0, v.r, -alpha, v.q, 0.0, nullptr, n, st));
        SGN_CUDA(apply_hw64(c, v.s, v.r, 1, !adj, nullptr, st));
        SGN_CHECK(gram<double2>(W, v.r, 2, v.r, 2, G));
        ++it;
        rn = std::sqrt(std::max(G[0].real(), 0.0));
        const double gnew = G[3].real();
        if (rn <= tol * bn) break;
        const double beta = gnew / gamma;
        gamma = gnew;
        SGN_CUDA(axpby3<double2>(v.p, 1.0, v.s, beta, v.p, 0.0, nullptr, n, st));
    }
    *its = it;
    *relres = rn / bn;
    return SGN_OK;
}

// Orthonormalise the columns of the p x k host matrix Y (row-major) in place by
// two classical Gram-Schmidt passes.
void orth_host(int p, int k, std::vector<cd>& Y) {
    for (int j = 0; j < k; ++j)
        for (int pass = 0; pass < 2; ++pass) {
            for (int l = 0; l < j; ++l) {
                cd h = 0;
                for (int i = 0; i < p; ++i) h += std::conj(Y[(size_t)i * k + l]) * Y[(size_t)i * k + j];
                for (int i = 0; i < p; ++i) Y[(size_t)i * k + j] -= h * Y[(size_t)i * k + l];
            }
            double nr = 0;
            for (int i = 0; i < p; ++i) nr += std::norm(Y[(size_t)i * k + j]);
            nr = std::sqrt(nr);
            for (int i = 0; i < p; ++i) Y[(size_t)i * k + j] /= nr;
        }
}

// The `want` eigenvectors of A (A^dag with adj) of smallest |lambda| into out
// (want FP64 fields, unit norm, not yet split by a Rayleigh-Ritz step with A):
// Ritz vectors of A^{-1} whose relative residual ||A^{-1} y - theta y|| / |theta|
// is below tolB.
int inverse_arnoldi(sgn_ctx* c, bool adj, int want, double tolB, uint64_t seed, double2* out) {
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    const int pmax = std::min(100, std::max(want + 24, 2 * want));
    const int keep = std::min(pmax - 12, want + (pmax - want) / 2);
    const double inner = std::max(1e-14, 0.1 * tolB);
    Work W;
    SGN_CHECK(setup(W, c, pmax + 1, sizeof(double2), reduce_blocks<double2>(n), 2));
    DevBuf cb;
    int rc = dev_alloc(c, cb, sizeof(double2) * (size_t)n * 5);
    if (rc != SGN_OK) {
        dev_free(c, W.buf);
        return rc;
    }
    double2* V = reinterpret_cast<double2*>(W.blk[0]);
    double2* T = reinterpret_cast<double2*>(W.blk[1]);
    double2* cbp = reinterpret_cast<double2*>(cb.p);
    const CglsVecs cv{cbp, cbp + n, cbp + 2 * n, cbp + 3 * n, cbp + 4 * n};
    auto fail_out = [&](int code) {
        dev_free(c, cb);
        dev_free(c, W.buf);
        return code;
    };
#define INV_CHECK(call)                    \
    do {                                   \
        int _r = (call);                   \
        if (_r != SGN_OK) return fail_out(_r); \
    } while (0)
#define INV_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t _e = (call);                                                        \
        if (_e != cudaSuccess) {                                                        \
            set_error(std::string("deflation set-up: ") + cudaGetErrorString(_e));      \
            return fail_out(SGN_ERR_CUDA);                                              \
        }                                                                               \
    } while (0)
    std::vector<cd> G, h1, h2;
    INV_CUDA(random_fill<double2>(V, n, seed, st));
    INV_CHECK(gram<double2>(W, V, 1, V, 1, G));
    INV_CUDA(axpby3<double2>(V, 1.0 / std::sqrt(G[0].real()), V, 0.0, V, 0.0, nullptr, n, st));
    std::vector<cd> H((size_t)(pmax + 1) * pmax, 0.0);  // Krylov decomposition A^{-1} V_p = V_{p+1} H
    int k = 0;
    const int max_cg = 20000;
    long long cg_total = 0;
    for (int restart = 0; restart < 60; ++restart) {
        for (int j = k; j < pmax; ++j) {
            double2* vj = V + (size_t)j * n;
            int its = 0;
            double rel = 0;
            INV_CHECK(cgls(W, adj, vj, cv, inner, max_cg, &its, &rel));
            cg_total += its;
            if (!(rel <= 100 * inner)) {
                set_error("deflation set-up: CGLS for A^{-1} did not converge (relative residual " +
                          std::to_string(rel) + ")");
                return fail_out(SGN_ERR_DEFLATION);
            }
            double2* w = cv.x;
            // two classical Gram-Schmidt passes against v_0 .. v_j
            INV_CHECK(gram<double2>(W, V, j + 1, w, 1, h1));
            INV_CHECK(combine<double2>(W, V, j + 1, h1, 1, T));
            INV_CUDA(axpby3<double2>(w, 1.0, w, -1.0, T, 0.0, nullptr, n, st));
            INV_CHECK(gram<double2>(W, V, j + 1, w, 1, h2));
            INV_CHECK(combine<double2>(W, V, j + 1, h2, 1, T));
            INV_CUDA(axpby3<double2>(w, 1.0, w, -1.0, T, 0.0, nullptr, n, st));
            for (int i = 0; i <= j; ++i) H[(size_t)i * pmax + j] += h1[i] + h2[i];
            INV_CHECK(gram<double2>(W, w, 1, w, 1, G));
            const double nrm = std::sqrt(std::max(G[0].real(), 0.0));
            if (!(nrm > 0) || !std::isfinite(nrm)) {
                set_error("deflation set-up: shift-invert Arnoldi broke down");
                return fail_out(SGN_ERR_DEFLATION);
            }
            H[(size_t)(j + 1) * pmax + j] = nrm;
            INV_CUDA(axpby3<double2>(V + (size_t)(j + 1) * n, 1.0 / nrm, w, 0.0, w, 0.0, nullptr, n, st));
        }
        // Ritz pairs of the p x p top block, largest |theta| first
        std::vector<cd> Hp((size_t)pmax * pmax), th, X;
        for (int i = 0; i < pmax; ++i)
            for (int j = 0; j < pmax; ++j) Hp[(size_t)i * pmax + j] = H[(size_t)i * pmax + j];
        if (dense_eig(pmax, Hp, th, X)) {
            set_error("deflation set-up: Arnoldi eigendecomposition failed");
            return fail_out(SGN_ERR_DEFLATION);
        }
        std::vector<int> ord(pmax);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return std::abs(th[a]) > std::abs(th[b]); });
        // residual of Ritz pair (theta, V y): |h_{p+1,p}| |e_p^T y| / (||y|| |theta|); the
        // bottom row of H carries the coupling (one entry after an Arnoldi step, a full
        // row right after a thick restart with no step taken -- never the case here)
        double worst = 0;
        const cd* hrow = &H[(size_t)pmax * pmax];
        for (int t = 0; t < want; ++t) {
            const int i = ord[t];
            double yn = 0;
            cd e = 0;
            for (int r = 0; r < pmax; ++r) {
                yn += std::norm(X[(size_t)r * pmax + i]);
                e += hrow[r] * X[(size_t)r * pmax + i];
            }
            worst = std::max(worst, std::abs(e) / (std::sqrt(yn) * std::abs(th[i])));
        }
        if (debug_on())
            fprintf(stderr, "[sgn eig inv %s] restart %d worst %.3e |theta| %.4e..%.4e cgls its %lld\n",
                    adj ? "left" : "right", restart, worst, std::abs(th[ord[0]]), std::abs(th[ord[want - 1]]),
                    cg_total);
        const int nk = worst <= tolB ? want : keep;
        // Q = orthonormalised Ritz coefficient vectors of the nk largest
        std::vector<cd> Q((size_t)pmax * nk);
        for (int r = 0; r < pmax; ++r)
            for (int t = 0; t < nk; ++t) Q[(size_t)r * nk + t] = X[(size_t)r * pmax + ord[t]];
        if (worst <= tolB) {  // the Ritz vectors themselves (unit norm)
            for (int t = 0; t < nk; ++t) {
                double yn = 0;
                for (int r = 0; r < pmax; ++r) yn += std::norm(Q[(size_t)r * nk + t]);
                yn = std::sqrt(yn);
                for (int r = 0; r < pmax; ++r) Q[(size_t)r * nk + t] /= yn;
            }
            INV_CHECK(combine<double2>(W, V, pmax, Q, want, T));
            INV_CUDA(cudaMemcpyAsync(out, T, sizeof(double2) * (size_t)want * n, cudaMemcpyDeviceToDevice, st));
            INV_CUDA(cudaStreamSynchronize(st));
            if (debug_on())
                fprintf(stderr, "[sgn eig inv] converged after %d restarts, %lld CGLS steps\n", restart, cg_total);
            dev_free(c, cb);
            dev_free(c, W.buf);
            return SGN_OK;
        }
        orth_host(pmax, nk, Q);
        // V_new = V_p Q, v_new[nk] = v_{p}; H_new = [Q^dag H_p Q ; h_{p+1}^T Q]
        INV_CHECK(combine<double2>(W, V, pmax, Q, nk, T));
        INV_CUDA(cudaMemcpyAsync(V + (size_t)nk * n, V + (size_t)pmax * n, sizeof(double2) * n,
                                 cudaMemcpyDeviceToDevice, st));
        INV_CUDA(cudaMemcpyAsync(V, T, sizeof(double2) * (size_t)nk * n, cudaMemcpyDeviceToDevice, st));
        std::vector<cd> HQ((size_t)pmax * nk, 0.0), Hn((size_t)(pmax + 1) * pmax, 0.0);
        for (int i = 0; i < pmax; ++i)
            for (int t = 0; t < nk; ++t) {
                cd acc = 0;
                for (int r = 0; r < pmax; ++r) acc += H[(size_t)i * pmax + r] * Q[(size_t)r * nk + t];
                HQ[(size_t)i * nk + t] = acc;
            }
        for (int a = 0; a < nk; ++a)
            for (int t = 0; t < nk; ++t) {
                cd acc = 0;
                for (int i = 0; i < pmax; ++i) acc += std::conj(Q[(size_t)i * nk + a]) * HQ[(size_t)i * nk + t];
                Hn[(size_t)a * pmax + t] = acc;
            }
        for (int t = 0; t < nk; ++t) {
            cd acc = 0;
            for (int r = 0; r < pmax; ++r) acc += hrow[r] * Q[(size_t)r * nk + t];
            Hn[(size_t)nk * pmax + t] = acc;
        }
        H.swap(Hn);
        k = nk;
    }
#undef INV_CHECK
#undef INV_CUDA
    set_error("deflation set-up: shift-invert Arnoldi did not converge");
    return fail_out(SGN_ERR_DEFLATION);
}

// One side: `want` eigenpairs of A (adj = false) or A^dag (adj = true) into V64 (want fields, FP64).
// Eigenpairs of A from `want` fields F (FP64, in block 4 of W64) spanning an
// invariant subspace: one Rayleigh-Ritz step with A; accepted when every relative
// residual is below tol.
int finish_side(Work& W64, bool adj, int want, double tol, double2* V64, std::vector<cd>& lam, bool* ok) {
    sgn_ctx* c = W64.c;
    double2* F = reinterpret_cast<double2*>(W64.blk[4]);
    Ritz ra;
    SGN_CHECK(svqb_final(W64, F, want, adj, ra));
    double worst = 0;
    for (int j = 0; j < want; ++j) worst = std::max(worst, ra.res[j]);
    if (debug_on()) fprintf(stderr, "[sgn eig] eigenpairs of A: worst relative residual %.3e\n", worst);
    *ok = worst <= tol;
    if (*ok) {
        SGN_CUDA(cudaMemcpyAsync(V64, F, sizeof(double2) * want * c->n, cudaMemcpyDeviceToDevice, c->work));
        SGN_CUDA(cudaStreamSynchronize(c->work));
        lam = ra.theta;
    }
    return SGN_OK;
}

// The shift-invert route for one side: Arnoldi on A^{-1}, then Rayleigh-Ritz with A.
int eig_side_inverse(sgn_ctx* c, bool adj, int want, double tol, uint64_t seed, double2* V64, std::vector<cd>& lam) {
    Work W64;
    SGN_CHECK(setup(W64, c, want, sizeof(double2), reduce_blocks<double2>(c->n)));
    double2* F = reinterpret_cast<double2*>(W64.blk[4]);
    // A-residual of a Ritz pair of A^{-1} with relative residual e is at most
    // e ||A|| / |lambda|: aim well below tol
    double tolB = tol / 100;
    int rc = SGN_OK;
    for (int attempt = 0; attempt < 3; ++attempt) {
        rc = inverse_arnoldi(c, adj, want, tolB, seed ^ 0x1f1fULL, F);
        if (rc != SGN_OK) break;
        bool ok = false;
        rc = finish_side(W64, adj, want, tol, V64, lam, &ok);
        if (rc != SGN_OK || ok) break;
        tolB /= 100;
        rc = SGN_ERR_DEFLATION;
        set_error("deflation set-up: eigenpairs of A did not reach the tolerance");
    }
    dev_free(c, W64.buf);
    return rc;
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
    int rc = spectrum_height2<float2>(W, adj, 200, seed ^ 0xa5a5ULL, &height);
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
    double worst32 = 0;
    for (int j = 0; j < want; ++j) worst32 = std::max(worst32, rz.res[j]);
    if (!(worst32 < 0.5)) {
        // the polynomial filter made no headway: no polynomial in A^2 separates the
        // wanted eigenvalues here
        if (debug_on()) fprintf(stderr, "[sgn eig] FP32 filter ended at %.3e: shift-invert Arnoldi\n", worst32);
        dev_free(c, W.buf);
        return eig_side_inverse(c, adj, want, tol, seed, V64, lam);
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
    if (worst32 <= 10 * tol) {  // a loose tolerance the FP32 phase may already meet
        double2* F = reinterpret_cast<double2*>(W64.blk[4]);
        SGN_CUDA(cudaMemcpyAsync(F, Y64, sizeof(double2) * want * c->n, cudaMemcpyDeviceToDevice, st));
        bool ok = false;
        rc = finish_side(W64, adj, want, tol, V64, lam, &ok);
        if (rc != SGN_OK || ok) {
            dev_free(c, W64.buf);
            return rc;
        }
    }
    // FP64: converge the A^2 subspace, then split it with one Rayleigh-Ritz step on A
    double tol2 = tol / 10;
    for (int attempt = 0; attempt < 4 && rc == SGN_OK; ++attempt) {
        rc = iterate<double2>(W64, adj, Y64, want, tol2, 40, rz, attempt == 0, false, &its);
        if (rc == SGN_ERR_DEFLATION && W64.weak) {  // the filter stalled: shift-invert instead
            if (debug_on()) fprintf(stderr, "[sgn eig] FP64 filter stalled: shift-invert Arnoldi\n");
            dev_free(c, W64.buf);
            return eig_side_inverse(c, adj, want, tol, seed, V64, lam);
        }
        if (rc != SGN_OK) break;
        double2* F = reinterpret_cast<double2*>(W64.blk[4]);
        SGN_CUDA(cudaMemcpyAsync(F, Y64, sizeof(double2) * want * c->n, cudaMemcpyDeviceToDevice, st));
        bool ok = false;
        rc = finish_side(W64, adj, want, tol, V64, lam, &ok);
        if (rc != SGN_OK) break;
        if (ok) {
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
    // the inverse iteration's GMRES engines (q columns each) are not needed by the solves
    release_engines(c);
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
    c->deflation_stale = false;
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
