// Restarted LR-deflated multishift FOM, Algorithm 1 ("FOM-LR(m,k)"), on the
// GPU.  The s shifted systems of eq. (2.2) are read with t^2 as in eq. (6.2):
// (A^2 - sigma_i) x_i = b~ with b~ = A (I - P) b, so one Arnoldi process on
// A^2 serves all shifts (shift invariance, Sec. 2) and every restart keeps the
// residuals collinear (eq. (3.1)).
//
// Host orchestration.  Every scalar of the method (Hessenberg entries, norms,
// collinearity factors, convergence flags) lives on the device, so a restart
// cycle -- k Arnoldi steps, the shifted solves, the update, the projection
// step and the restart -- is a fixed launch sequence.  It is captured once as
// a CUDA graph and replayed; the host reads back only the per-column
// convergence flags between cycles.  Columns (right-hand sides) run in
// lockstep with separate Krylov spaces; a converged column skips its work.
#include "ctx.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

namespace sgn {

int dev_alloc(sgn_ctx* c, DevBuf& b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return SGN_OK;
    dev_free(c, b);
    if (bytes == 0) return SGN_OK;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->user);
        if (!p) {
            set_error("device allocation of " + std::to_string(bytes) + " bytes failed (caller allocator)");
            return SGN_ERR_ALLOC;
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
            return SGN_ERR_ALLOC;
        }
    }
    b.p = p;
    b.bytes = bytes;
    return SGN_OK;
}

void dev_free(sgn_ctx* c, DevBuf& b) {
    if (!b.p) return;
    if (c->free_)
        c->free_(b.p, b.bytes, c->user);
    else
        cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

void fill_fp32_coefficients(StencilParams& p) {
    for (int d = 0; d < 3; ++d) p.div[d] = FastDiv((uint32_t)p.L[d]);
    p.diag32 = (float)p.diag;
    p.diag_lo = (float)(p.diag - (double)p.diag32);
    for (int d = 0; d < 4; ++d) {
        p.cf32[d] = (float)p.cf[d];
        p.cb32[d] = (float)p.cb[d];
        p.cf_lo[d] = (float)(p.cf[d] - (double)p.cf32[d]);
        p.cb_lo[d] = (float)(p.cb[d] - (double)p.cb32[d]);
    }
}

StencilParams stencil_params(const sgn_ctx* c, bool adjoint) {
    StencilParams p{};
    for (int d = 0; d < 4; ++d) {
        p.L[d] = c->dims[d];
        p.ap[d] = c->ap[d];
        p.cf[d] = -0.5;
        p.cb[d] = -0.5;
    }
    const double mu = adjoint ? -c->mu : c->mu;
    p.cf[3] = -0.5 * std::exp(mu);
    p.cb[3] = -0.5 * std::exp(-mu);
    p.vol = c->vol;
    p.stride_rhs = c->n;
    p.diag = 4.0 + c->mass;
    fill_fp32_coefficients(p);
    return p;
}

namespace {
StencilShape shape_for(const sgn_ctx* c, int prec, int ncol) {
    auto it = c->shapes.find(prec * 4096 + ncol);
    return it == c->shapes.end() ? StencilShape{} : it->second;
}
}  // namespace

cudaError_t apply_hw64(const sgn_ctx* c, double2* out, const double2* in, int ncol, bool adjoint, const int* skip,
                       cudaStream_t st) {
    return launch_hw_f64(out, in, reinterpret_cast<const double2*>(c->U64.p), ncol, stencil_params(c, adjoint), skip,
                         st, shape_for(c, 0, ncol));
}

cudaError_t apply_hw32(const sgn_ctx* c, float2* out, const float2* in, int ncol, bool adjoint, const int* skip,
                       cudaStream_t st, bool fp32_links) {
    StencilParams p = stencil_params(c, adjoint);
    const int prec = fp32_links ? 1 : stencil_prec32(c);
    if (prec == 2)
        return launch_hw_f32_bf16links(out, in, reinterpret_cast<const __nv_bfloat162*>(c->U16.p), ncol, p, skip, st,
                                       shape_for(c, prec, ncol));
    if (prec == 3)
        return launch_hw_f32_f16links(out, in, reinterpret_cast<const __half2*>(c->UH.p), ncol, p, skip, st,
                                      shape_for(c, prec, ncol));
    return launch_hw_f32(out, in, reinterpret_cast<const float2*>(c->U32.p), ncol, p, skip, st,
                         shape_for(c, prec, ncol));
}

int tune_stencil(sgn_ctx* c, int prec, int ncol, void* in, void* out) {
    const int key = prec * 4096 + ncol;
    if (c->shapes.count(key)) return SGN_OK;
    static const bool off = [] {
        const char* s = getenv("SGN_NO_TUNE");
        return s && s[0] == '1';
    }();
    if (off) {
        c->shapes[key] = StencilShape{};
        return SGN_OK;
    }
    // SGN_STENCIL_SHAPE="sx,rb,nr[,pipe]" fixes the shape of every stencil launch (checked at launch)
    if (const char* fix = getenv("SGN_STENCIL_SHAPE")) {
        StencilShape sh;
        if (sscanf(fix, "%d,%d,%d,%d", &sh.sx, &sh.rb, &sh.nr, &sh.pipe) >= 3) {
            c->shapes[key] = sh;
            return SGN_OK;
        }
    }
    cudaStream_t st = c->work;
    const StencilParams p = stencil_params(c, false);
    std::vector<StencilShape> cands;
    for (int pipe = 0; pipe <= (prec == 0 ? 0 : 3); ++pipe)
        for (int nr : {1, 2, 3}) {
            if (pipe == 4) continue;  // the colour-split kernel has its own shapes below
            if (nr > ncol || (prec == 0 && nr > 1) || (pipe == 1 && nr > 2) || (pipe >= 2 && nr != 2)) continue;
            const int groups = (ncol + nr - 1) / nr;
            const int maxt = nr == 1 && !pipe ? 384 : 256;
            for (int rb : {1, 2, 3, 4, 6, 8, 12, 16}) {
                if (rb > groups) continue;
                for (int sx : {32, 64, 128, 256})
                    if (sx * rb <= maxt && sx * rb >= 64) cands.push_back({sx, rb, nr, pipe});
            }
        }
    if (prec != 0)  // colour-split kernel: sg site groups of 10 sites x fw fields per CTA (<= 8 warps)
        for (int fw : {1, 2, 3, 4, 6, 8})
            for (int sg : {1, 2, 4, 8})
                if (fw <= ncol && sg * fw <= 8 && sg * fw >= 2) cands.push_back({sg, fw, 1, 4});
    if (cands.empty()) cands.push_back({});
    auto run = [&](StencilShape sh) -> cudaError_t {
        if (prec == 0)
            return launch_hw_f64(reinterpret_cast<double2*>(out), reinterpret_cast<const double2*>(in),
                                 reinterpret_cast<const double2*>(c->U64.p), ncol, p, nullptr, st, sh);
        if (prec == 2)
            return launch_hw_f32_bf16links(reinterpret_cast<float2*>(out), reinterpret_cast<const float2*>(in),
                                           reinterpret_cast<const __nv_bfloat162*>(c->U16.p), ncol, p, nullptr, st,
                                           sh);
        if (prec == 3)
            return launch_hw_f32_f16links(reinterpret_cast<float2*>(out), reinterpret_cast<const float2*>(in),
                                          reinterpret_cast<const __half2*>(c->UH.p), ncol, p, nullptr, st, sh);
        return launch_hw_f32(reinterpret_cast<float2*>(out), reinterpret_cast<const float2*>(in),
                             reinterpret_cast<const float2*>(c->U32.p), ncol, p, nullptr, st, sh);
    };
    float best = 1e30f;
    StencilShape pick{};
    const long long l0 = g_launches;
    for (const StencilShape& sh : cands) {
        for (int w = 0; w < 2; ++w) SGN_CUDA(run(sh));
        SGN_CUDA(cudaEventRecord(c->ev_k0, st));
        for (int r = 0; r < 3; ++r) SGN_CUDA(run(sh));
        SGN_CUDA(cudaEventRecord(c->ev_k1, st));
        SGN_CUDA(cudaEventSynchronize(c->ev_k1));
        float ms = 0;
        SGN_CUDA(cudaEventElapsedTime(&ms, c->ev_k0, c->ev_k1));
        if (ms < best) {
            best = ms;
            pick = sh;
        }
    }
    g_launches = l0;  // tuning launches are not part of the solve
    c->shapes[key] = pick;
    static const bool dbg = [] {
        const char* s = getenv("SGN_DEBUG");
        return s && s[0] == '1';
    }();
    if (dbg)
        fprintf(stderr, "[sgn tune] stencil prec %d ncol %d -> sx %d rb %d nr %d pipe %d (%.3f ms / 3)\n", prec, ncol,
                pick.sx, pick.rb, pick.nr, pick.pipe, best);
    return SGN_OK;
}

namespace {

template <class T>
cudaError_t apply_hw(const sgn_ctx* c, T* out, const T* in, int ncol, bool adjoint, const int* skip,
                     cudaStream_t st);
template <>
cudaError_t apply_hw<double2>(const sgn_ctx* c, double2* out, const double2* in, int ncol, bool adjoint,
                              const int* skip, cudaStream_t st) {
    return apply_hw64(c, out, in, ncol, adjoint, skip, st);
}
template <>
cudaError_t apply_hw<float2>(const sgn_ctx* c, float2* out, const float2* in, int ncol, bool adjoint, const int* skip,
                             cudaStream_t st) {
    return apply_hw32(c, out, in, ncol, adjoint, skip, st);
}

#define CU(x)                                     \
    do {                                          \
        cudaError_t _e = (x);                     \
        if (_e != cudaSuccess) return _e;         \
    } while (0)

uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    return h;
}

// Everything a captured cycle depends on besides the engine's own buffers.
struct CycleArgs {
    bool adjoint = false;
    const void* L = nullptr;  // deflation blocks in the storage precision (n x m)
    const void* R = nullptr;
    int m = 0;
    int project = 1;
    double2* xacc = nullptr;  // FP64 accumulator of x (combined), may be null
    int64_t xsr = 0;
    double2* xs = nullptr;    // FP64 per-shift iterates, may be null
    int64_t xs_shift = 0, xs_col = 0;
    bool gmres = false;       // minimal-residual restarts (one shift per column, FP64 engines)
    bool op_a = false;        // Krylov space of A itself (the split form), else of A^2
};

uint64_t cycle_key(const sgn_ctx* c, const Engine& E, const CycleArgs& a) {
    uint64_t h = 1469598103934665603ULL;
    auto mixd = [&](double d) {
        uint64_t u;
        std::memcpy(&u, &d, 8);
        h = mix(h, u);
    };
    h = mix(h, a.adjoint);
    h = mix(h, (uint64_t)(uintptr_t)a.L);
    h = mix(h, (uint64_t)(uintptr_t)a.R);
    h = mix(h, a.m);
    h = mix(h, a.project);
    h = mix(h, (uint64_t)(uintptr_t)a.xacc);
    h = mix(h, a.xsr);
    h = mix(h, (uint64_t)(uintptr_t)a.xs);
    h = mix(h, a.xs_shift);
    h = mix(h, a.xs_col);
    h = mix(h, a.gmres);
    h = mix(h, a.op_a);
    h = mix(h, (uint64_t)(uintptr_t)c->U64.p);
    h = mix(h, (uint64_t)(uintptr_t)c->U32.p);
    h = mix(h, (uint64_t)(uintptr_t)c->U16.p);
    h = mix(h, (uint64_t)(uintptr_t)c->UH.p);
    h = mix(h, c->link_storage);
    mixd(c->mu);
    mixd(c->mass);
    for (int d = 0; d < 4; ++d) h = mix(h, c->ap[d]);
    mixd(E.S.tol);
    h = mix(h, c->timing);
    return h;
}

// Event pair around one launch of a timed kernel class (only while capturing a
// cycle with timing on); the pair is replayed with the graph.
struct Timer {
    const sgn_ctx* c;
    Engine& E;
    cudaStream_t st;
    int idx = -1;
    Timer(const sgn_ctx* c_, Engine& E_, cudaStream_t st_) : c(c_), E(E_), st(st_) {}
    cudaError_t begin(int cls, double bytes) {
        if (!c->timing) return cudaSuccess;
        idx = (int)E.tmarks.size();
        while ((int)E.tev.size() < 2 * (idx + 1)) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return e;
            E.tev.push_back(ev);
        }
        E.tmarks.emplace_back(cls, bytes);
        // external: recorded as an event node of the captured graph (a plain record
        // inside a capture only orders the stream and records nothing)
        return cudaEventRecordWithFlags(E.tev[2 * idx], st, cudaEventRecordExternal);
    }
    cudaError_t end() {
        if (!c->timing) return cudaSuccess;
        return cudaEventRecordWithFlags(E.tev[2 * idx + 1], st, cudaEventRecordExternal);
    }
};

bool debug_log() {
    static const bool v = [] {
        const char* s = getenv("SGN_DEBUG");
        return s && s[0] == '1';
    }();
    return v;
}

bool use_cgs2() {
    static const bool v = [] {
        const char* s = getenv("SGN_ORTHO");
        return s && std::string(s) == "cgs2";
    }();
    return v;
}

// One restart cycle of Algorithm 1, Arnoldi by delayed CGS2: the second
// projection of each new basis vector is done in the next step's single fused
// reduction, so every step reads the basis twice (one reduction sweep, one
// update sweep) instead of three times.  On entry V[0] holds the unnormalised
// restart vector; step 0 normalises it and records beta.
template <class T>
cudaError_t cycle_dcgs(const sgn_ctx* c, Engine& E, const CycleArgs& a, cudaStream_t st) {
    const int64_t n = E.n;
    const int ncol = E.ncol, k = E.k;
    T* V = reinterpret_cast<T*>(E.V);
    T* w = reinterpret_cast<T*>(E.w);
    T* t = reinterpret_cast<T*>(E.t);
    const int64_t sj = (int64_t)ncol * n, sr = n;
    const Reduce rd{E.partial, E.nblk, E.rstride};
    const DevState& S = E.S;
    const Basis<T> VB{V, sj, sr};
    const double fb = (double)n * sizeof(T) * ncol;            // one field per column
    const double stb = (double)c->vol * 4 * 9 * sizeof(T) + 2 * fb;  // links once, in and out once
    Timer tm(c, E, st);
    for (int j = 0; j < k; ++j) {
        // z = A^2 u_j (u_j: candidate for v_j, once orthogonalised); z = A u_j in the split form
        CU(tm.begin(0, stb));
        CU(apply_hw<T>(c, a.op_a ? w : t, V + j * sj, ncol, a.adjoint, S.skip, st));
        CU(tm.end());
        if (!a.op_a) {
            CU(tm.begin(0, stb));
            CU(apply_hw<T>(c, w, t, ncol, a.adjoint, S.skip, st));
            CU(tm.end());
        }
        CU(tm.begin(1, (j + 2) * fb));
        CU(dcgs_dots<T>(VB, j, V + j * sj, w, sr, n, ncol, rd, S.skip, st));
        CU(tm.end());
        CU(tm.begin(3, (double)(2 * j + 3) * E.nblk * sizeof(double2) * ncol));
        CU(reduce(rd, 2 * j + 3, ncol, RM_DCGS, j, S, nullptr, st));
        CU(tm.end());
        CU(tm.begin(2, (j + 4) * fb));
        CU(dcgs_update<T>(VB, j, S.red, S.rstride, V + j * sj, w, V + (j + 1) * sj, sr, n, ncol, S.skip, st));
        CU(tm.end());
    }
    // closing pass: second projection of v_k
    CU(tm.begin(1, (k + 1) * fb));
    CU(dcgs_dots<T>(VB, k, V + k * sj, nullptr, sr, n, ncol, rd, S.skip, st));
    CU(tm.end());
    CU(tm.begin(3, (double)(k + 1) * E.nblk * sizeof(double2) * ncol));
    CU(reduce(rd, k + 1, ncol, RM_DCGS_FINAL, k, S, nullptr, st));
    CU(tm.end());
    CU(tm.begin(2, (k + 2) * fb));
    CU(dcgs_update<T>(VB, k, S.red, S.rstride, V + k * sj, nullptr, nullptr, sr, n, ncol, S.skip, st));
    CU(tm.end());
    if (a.gmres) {
        CU(shifted_lsq(S, ncol, st));
    } else {
        CU(shifted_solves(S, ncol, st));
    }
    CU(combine_shifts(S, ncol, st));
    if (a.xacc) CU(update_x<T>(VB, k, S.coef, S.rstride, a.xacc, a.xsr, n, ncol, S.done, S.kk, st));
    if (a.xs) {
        // the basis once (the shift groups of a tile share it through L2), every per-shift
        // iterate read and written (FP64)
        CU(tm.begin(4, (double)k * fb + 2.0 * E.s * ncol * n * sizeof(double2)));
        CU(update_shifts<T>(VB, k, S.y, E.s, k, a.xs, a.xs_shift, a.xs_col, n, ncol, S.done, S.kk, st));
        CU(tm.end());
    }
    T* Vk = V + k * sj;
    if (a.gmres) {  // the minimal residual r = V_{k+1} c becomes the restart vector
        T* tt = reinterpret_cast<T*>(E.t);
        CU(cudaMemsetAsync(tt, 0, sizeof(T) * (size_t)ncol * n, st));
        if constexpr (sizeof(T) == sizeof(double2)) {
            CU(update_x<T>(VB, k + 1, S.gres, k + 1, reinterpret_cast<double2*>(tt), n, n, ncol, S.done, nullptr, st));
        } else {  // FP32 basis: (0 - V c) * (-1), accumulated in FP32 like every basis update
            CU(maxpy_scale<T>(VB, k + 1, S.gres, k + 1, tt, n, tt, n, E.neg1, n, ncol, S.done, st));
        }
        CU(cudaMemcpyAsync(Vk, tt, sizeof(T) * (size_t)ncol * n, cudaMemcpyDeviceToDevice, st));
    }
    if (a.project && a.m > 0) {
        const Basis<T> LB{reinterpret_cast<const T*>(a.L), n, 0};
        const Basis<T> RB{reinterpret_cast<const T*>(a.R), n, 0};
        CU(mdot<T>(LB, a.m, Vk, sr, n, ncol, rd, 0, S.skip, st));
        CU(reduce(rd, a.m, ncol, RM_STORE, 0, S, nullptr, st));
        CU(maxpy_scale<T>(RB, a.m, S.red, S.rstride, Vk, sr, Vk, sr, nullptr, n, ncol, S.skip, st));
    }
    // convergence test on ||r||; r (unnormalised) becomes the next cycle's V[0]
    CU(mdot<T>(VB, 0, Vk, sr, n, ncol, rd, 1, S.skip, st));
    CU(reduce(rd, 1, ncol, RM_BETA_RESTART, 0, S, nullptr, st));
    CU(maxpy_scale<T>(VB, 0, S.red, S.rstride, Vk, sr, V, sr, nullptr, n, ncol, S.skip, st));
    return cudaSuccess;
}

// One restart cycle of Algorithm 1 for all columns, Arnoldi by CGS2 in three
// passes per step (kept for comparison; SGN_ORTHO=cgs2).
template <class T>
cudaError_t cycle(const sgn_ctx* c, Engine& E, const CycleArgs& a, cudaStream_t st) {
    if (!use_cgs2()) return cycle_dcgs<T>(c, E, a, st);
    const int64_t n = E.n;
    const int ncol = E.ncol, k = E.k;
    T* V = reinterpret_cast<T*>(E.V);
    T* w = reinterpret_cast<T*>(E.w);
    T* t = reinterpret_cast<T*>(E.t);
    const int64_t sj = (int64_t)ncol * n, sr = n;
    const Reduce rd{E.partial, E.nblk, E.rstride};
    const DevState& S = E.S;
    const Basis<T> VB{V, sj, sr};
    for (int j = 0; j < k; ++j) {
        // w = A^2 v_j
        if (a.op_a) {
            CU(apply_hw<T>(c, w, V + j * sj, ncol, a.adjoint, S.skip, st));
        } else {
            CU(apply_hw<T>(c, t, V + j * sj, ncol, a.adjoint, S.skip, st));
            CU(apply_hw<T>(c, w, t, ncol, a.adjoint, S.skip, st));
        }
        // CGS2: h1 = V^dag w; w -= V h1, h2 = V^dag w; v_{j+1} = (w - V h2) / h_{j+1,j}
        CU(mdot<T>(VB, j + 1, w, sr, n, ncol, rd, 1, S.skip, st));
        CU(reduce(rd, j + 2, ncol, RM_H1, j, S, nullptr, st));
        CU(maxpy_mdot<T>(VB, j + 1, S.h1, S.rstride, w, sr, n, ncol, rd, S.skip, st));
        CU(reduce(rd, j + 2, ncol, RM_P2, j, S, nullptr, st));
        CU(maxpy_scale<T>(VB, j + 1, S.red, S.rstride, w, sr, V + (j + 1) * sj, sr, S.scale, n, ncol, S.skip, st));
    }
    // y_i = beta rho_i (H_k - sigma_i)^{-1} e_1, rho_i update, c = sum omega_i y_i
    CU(shifted_solves(S, ncol, st));
    CU(combine_shifts(S, ncol, st));
    // x += V_k c  (and x_i += V_k y_i)
    if (a.xacc) CU(update_x<T>(VB, k, S.coef, S.rstride, a.xacc, a.xsr, n, ncol, S.done, S.kk, st));
    if (a.xs) CU(update_shifts<T>(VB, k, S.y, E.s, k, a.xs, a.xs_shift, a.xs_col, n, ncol, S.done, S.kk, st));
    // r = v_{k+1}; projection step r = (I - P) r
    T* Vk = V + k * sj;
    if (a.project && a.m > 0) {
        const Basis<T> LB{reinterpret_cast<const T*>(a.L), n, 0};
        const Basis<T> RB{reinterpret_cast<const T*>(a.R), n, 0};
        CU(mdot<T>(LB, a.m, Vk, sr, n, ncol, rd, 0, S.skip, st));
        CU(reduce(rd, a.m, ncol, RM_STORE, 0, S, nullptr, st));
        CU(maxpy_scale<T>(RB, a.m, S.red, S.rstride, Vk, sr, Vk, sr, nullptr, n, ncol, S.skip, st));
    }
    // beta = ||r||, convergence test, v_1 = r / beta
    CU(mdot<T>(VB, 0, Vk, sr, n, ncol, rd, 1, S.skip, st));
    CU(reduce(rd, 1, ncol, RM_BETA_RESTART, 0, S, nullptr, st));
    CU(maxpy_scale<T>(VB, 0, S.red, S.rstride, Vk, sr, V, sr, S.scale, n, ncol, S.skip, st));
    return cudaSuccess;
}

int get_engine(sgn_ctx* c, int ncol, int k, int s, int prec, Engine** out) {
    const uint64_t key = mix(mix(mix(mix((uint64_t)ncol, (uint64_t)k), (uint64_t)s), (uint64_t)prec),
                             (uint64_t)c->m);
    auto it = c->engines.find(key);
    if (it != c->engines.end()) {
        *out = it->second.get();
        return SGN_OK;
    }
    auto E = std::make_unique<Engine>();
    E->ncol = ncol;
    E->k = k;
    E->s = s;
    E->prec = prec;
    E->m = c->m;
    E->n = c->n;
    const size_t esz = prec == SGN_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    E->nblk = prec == SGN_PREC_FP64 ? wave_blocks<double2>(c->n, ncol) : wave_blocks<float2>(c->n, ncol);
    int rs = std::max(2 * k + 4, c->m + 1);
    E->rstride = (rs + 7) & ~7;
    const size_t nc = (size_t)ncol;
    const size_t field = (size_t)c->n * esz;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    size_t oV = take((size_t)(k + 1) * nc * field);
    size_t ow = take(nc * field);
    size_t ot = take(nc * field);
    size_t op = take(nc * E->rstride * (size_t)E->nblk * sizeof(double2));
    size_t oH = take(nc * (size_t)(k + 1) * k * sizeof(double2));
    size_t ored = take(nc * E->rstride * sizeof(double2));
    size_t oh1 = take(nc * E->rstride * sizeof(double2));
    size_t ocoef = take(nc * E->rstride * sizeof(double2));
    size_t oy = take(nc * (size_t)s * k * sizeof(double2));
    size_t orho = take(nc * (size_t)s * sizeof(double2));
    size_t od[5];
    for (int i = 0; i < 5; ++i) od[i] = take(nc * sizeof(double));
    size_t osig = take(nc * (size_t)s * sizeof(double));
    size_t oom = take(nc * (size_t)s * sizeof(double));
    size_t osim = take(nc * (size_t)s * sizeof(double));
    size_t oi[3];
    for (int i = 0; i < 3; ++i) oi[i] = take(nc * sizeof(int));
    size_t oerr = take(sizeof(int));
    size_t osums = take(nc * E->rstride * sizeof(double2));
    size_t ocnt = take(nc * sizeof(int));
    size_t ogres = take(nc * (size_t)(k + 1) * sizeof(double2));
    size_t oneg = take(nc * sizeof(double));
    size_t ocyc = take(sizeof(int));
    SGN_CHECK(dev_alloc(c, E->arena, off));
    char* base = reinterpret_cast<char*>(E->arena.p);
    E->V = base + oV;
    E->w = base + ow;
    E->t = base + ot;
    E->partial = reinterpret_cast<double2*>(base + op);
    DevState& S = E->S;
    S.H = reinterpret_cast<double2*>(base + oH);
    S.red = reinterpret_cast<double2*>(base + ored);
    S.h1 = reinterpret_cast<double2*>(base + oh1);
    S.coef = reinterpret_cast<double2*>(base + ocoef);
    S.y = reinterpret_cast<double2*>(base + oy);
    S.rho = reinterpret_cast<double2*>(base + orho);
    S.norm0 = reinterpret_cast<double*>(base + od[0]);
    S.scale = reinterpret_cast<double*>(base + od[1]);
    S.beta = reinterpret_cast<double*>(base + od[2]);
    S.bnorm = reinterpret_cast<double*>(base + od[3]);
    S.resest = reinterpret_cast<double*>(base + od[4]);
    E->sigma_dev = reinterpret_cast<double*>(base + osig);
    E->omega_dev = reinterpret_cast<double*>(base + oom);
    E->sigma_im_dev = reinterpret_cast<double*>(base + osim);
    S.sigma = E->sigma_dev;
    S.omega = E->omega_dev;
    S.sigma_im = E->sigma_im_dev;
    S.kk = reinterpret_cast<int*>(base + oi[0]);
    S.done = reinterpret_cast<int*>(base + oi[1]);
    S.skip = reinterpret_cast<int*>(base + oi[2]);
    S.err = reinterpret_cast<int*>(base + oerr);
    S.sums = reinterpret_cast<double2*>(base + osums);
    S.rcount = reinterpret_cast<int*>(base + ocnt);
    S.gres = reinterpret_cast<double2*>(base + ogres);
    S.kmax = k;
    S.s = s;
    S.rstride = E->rstride;
    S.bd_tol = prec == SGN_PREC_FP64 ? 1e-14 : 1e-6;
    E->neg1 = reinterpret_cast<double*>(base + oneg);
    E->cyc_dev = reinterpret_cast<int*>(base + ocyc);
    // zero the whole arena once so no kernel ever reads uninitialised memory
    SGN_CUDA(cudaMemsetAsync(E->arena.p, 0, off, c->work));
    {
        std::vector<double> m1(nc, -1.0);
        SGN_CUDA(cudaMemcpyAsync(E->neg1, m1.data(), nc * sizeof(double), cudaMemcpyHostToDevice, c->work));
        SGN_CUDA(cudaStreamSynchronize(c->work));  // m1 is released on return
    }
    SGN_CUDA(cudaHostAlloc(&E->h_done, nc * sizeof(int), cudaHostAllocDefault));
    SGN_CUDA(cudaHostAlloc(&E->h_resest, nc * sizeof(double), cudaHostAllocDefault));
    SGN_CUDA(cudaHostAlloc(&E->h_err, sizeof(int), cudaHostAllocDefault));
    SGN_CUDA(cudaHostAlloc(&E->h_kk, nc * sizeof(int), cudaHostAllocDefault));
    *out = E.get();
    c->engines[key] = std::move(E);
    return SGN_OK;
}

}  // namespace

void release_engines(sgn_ctx* c) {
    for (auto& kv : c->engines) {
        Engine& E = *kv.second;
        if (E.graph) cudaGraphExecDestroy(E.graph);
        if (E.loop) cudaGraphExecDestroy(E.loop);
        for (cudaEvent_t ev : E.tev) cudaEventDestroy(ev);
        dev_free(c, E.arena);
        if (E.h_done) cudaFreeHost(E.h_done);
        if (E.h_resest) cudaFreeHost(E.h_resest);
        if (E.h_err) cudaFreeHost(E.h_err);
        if (E.h_kk) cudaFreeHost(E.h_kk);
    }
    c->engines.clear();
    c->last_fp64 = nullptr;
}

namespace {

// End of one restart cycle inside the device loop (Algorithm 1's "while not all systems
// are converged"): count the cycle and keep looping unless every column has converged,
// the error word is set, or the cycle cap is reached.  One warp; the counter only grows,
// so the loop ends after at most max_cycles bodies.
__global__ void k_loop_decide(cudaGraphConditionalHandle h, const int* __restrict__ done, int ncol,
                              const int* __restrict__ err, int* __restrict__ cyc, int max_cycles) {
    bool all = true;
    for (int i = threadIdx.x; i < ncol; i += 32) all = all && done[i] != 0;
    all = __all_sync(0xffffffffu, all);
    if (threadIdx.x == 0) {
        const int cnum = *cyc + 1;
        *cyc = cnum;
        const bool stop = all || *err != 0 || cnum >= max_cycles;
        cudaGraphSetConditional(h, stop ? 0u : 1u);
    }
}

struct RunResult {
    int cycles = 0;
    int converged = 0;
    int breakdown = 0;
    int err = 0;
    double resmax = 0;
};

// Run restart cycles until every column has converged.  On entry V[0] holds
// the (unnormalised) first restart vector of every column and the shift
// tables of the engine are filled.
template <class T>
int run_engine(sgn_ctx* c, Engine& E, const CycleArgs& a, double tol, int max_cycles, RunResult* res) {
    cudaStream_t st = c->work;
    const int ncol = E.ncol;
    const int64_t n = E.n;
    E.S.tol = tol;
    SGN_CUDA(cudaMemsetAsync(E.S.done, 0, ncol * sizeof(int), st));
    SGN_CUDA(cudaMemsetAsync(E.S.skip, 0, ncol * sizeof(int), st));
    SGN_CUDA(cudaMemsetAsync(E.S.err, 0, sizeof(int), st));
    T* V = reinterpret_cast<T*>(E.V);
    const Reduce rd{E.partial, E.nblk, E.rstride};
    const Basis<T> VB{V, (int64_t)ncol * n, n};
    // beta = ||b~||, rho_i = 1, v_1 = b~ / beta
    SGN_CUDA(mdot<T>(VB, 0, V, n, n, ncol, rd, 1, nullptr, st));
    SGN_CUDA(reduce(rd, 1, ncol, RM_BETA_FIRST, 0, E.S, nullptr, st));
    if (use_cgs2())  // delayed CGS2 normalises the restart vector in its first step
        SGN_CUDA(maxpy_scale<T>(VB, 0, E.S.red, E.S.rstride, V, n, V, n, E.S.scale, n, ncol, E.S.skip, st));

    const uint64_t key = cycle_key(c, E, a);
    if (E.graph && E.graph_key != key) {
        cudaGraphExecDestroy(E.graph);
        E.graph = nullptr;
    }
    static const bool no_graph = [] {
        const char* s = getenv("SGN_NO_GRAPH");
        return s && s[0] == '1';
    }();
    if (!E.graph && !no_graph) {
        cudaGraph_t g = nullptr;
        E.tmarks.clear();
        SGN_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const long long before = g_launches;
        cudaError_t ce = cycle<T>(c, E, a, st);
        cudaError_t ee = cudaStreamEndCapture(st, &g);
        E.graph_kernels = g_launches - before;
        g_launches = before;  // capturing launches nothing
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            set_error(std::string("capturing the restart cycle failed: ") +
                      cudaGetErrorString(ce != cudaSuccess ? ce : ee));
            return SGN_ERR_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&E.graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            E.graph = nullptr;
            set_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
            return SGN_ERR_CUDA;
        }
        E.graph_key = key;
    }
    int cyc = 0;
    bool all_done = false;
    // The restart loop on the device: one graph launch runs cycles until every column has
    // converged (no host round trip per cycle).  Not with per-kernel timing (event nodes
    // are not allowed inside a conditional body) or the per-cycle debug log; if the runtime
    // refuses the conditional node, the host loop below runs instead.
    static const bool no_loop = [] {
        const char* s = getenv("SGN_HOST_LOOP");
        return s && s[0] == '1';
    }();
    if (E.graph && !c->timing && !debug_log() && !no_loop && !E.loop_unavailable) {
        const uint64_t lkey = mix(key, (uint64_t)max_cycles);
        if (E.loop && E.loop_key != lkey) {
            cudaGraphExecDestroy(E.loop);
            E.loop = nullptr;
        }
        if (!E.loop) {
            cudaGraph_t g = nullptr;
            cudaGraphConditionalHandle h = 0;
            cudaGraphNode_t node = nullptr;
            cudaGraphNodeParams cp{};
            cudaError_t e = cudaGraphCreate(&g, 0);
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
            if (e == cudaSuccess) {
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
            }
            if (e == cudaSuccess) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    const long long before = g_launches;
                    E.tmarks.clear();
                    cudaError_t ce = cycle<T>(c, E, a, st);
                    if (ce == cudaSuccess) {
                        k_loop_decide<<<1, 32, 0, st>>>(h, E.S.done, ncol, E.S.err, E.cyc_dev, max_cycles);
                        ce = cudaGetLastError();
                    }
                    g_launches = before;
                    cudaGraph_t cap = nullptr;
                    cudaError_t ee = cudaStreamEndCapture(st, &cap);
                    e = ce != cudaSuccess ? ce : ee;
                }
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&E.loop, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                E.loop = nullptr;
                E.loop_unavailable = true;
                cudaGetLastError();  // clear the refusal; the host loop takes over
                if (debug_log()) fprintf(stderr, "[sgn] device restart loop unavailable: %s\n", cudaGetErrorString(e));
            } else {
                E.loop_key = lkey;
            }
        }
        if (E.loop) {
            SGN_CUDA(cudaMemsetAsync(E.cyc_dev, 0, sizeof(int), st));
            SGN_CUDA(cudaGraphLaunch(E.loop, st));
            int ran = 0;
            SGN_CUDA(cudaMemcpyAsync(E.h_done, E.S.done, ncol * sizeof(int), cudaMemcpyDeviceToHost, st));
            SGN_CUDA(cudaMemcpyAsync(E.h_err, E.S.err, sizeof(int), cudaMemcpyDeviceToHost, st));
            SGN_CUDA(cudaMemcpyAsync(E.h_kk, E.cyc_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
            SGN_CUDA(cudaStreamSynchronize(st));
            ran = E.h_kk[0];
            count_launch((E.graph_kernels + 1) * (long long)ran);
            all_done = true;
            for (int i = 0; i < ncol; ++i) all_done = all_done && E.h_done[i];
            cyc = ran;
            goto finish;
        }
    }
    {
    // kernel timing: the bytes of a cycle count only the columns still active in it
    // (converged columns skip their work in every kernel)
    int active = ncol;
    if (c->timing) {
        SGN_CUDA(cudaMemcpyAsync(E.h_done, E.S.done, ncol * sizeof(int), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        active = 0;
        for (int i = 0; i < ncol; ++i) active += E.h_done[i] == 0;
    }
    for (; cyc < max_cycles; ++cyc) {
        if (E.graph) {
            SGN_CUDA(cudaGraphLaunch(E.graph, st));
            count_launch(E.graph_kernels);
        } else {
            E.tmarks.clear();
            SGN_CUDA(cycle<T>(c, E, a, st));
        }
        SGN_CUDA(cudaMemcpyAsync(E.h_done, E.S.done, ncol * sizeof(int), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaMemcpyAsync(E.h_err, E.S.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        if (c->timing)
            for (size_t i = 0; i < E.tmarks.size(); ++i) {
                float ms = 0;
                SGN_CUDA(cudaEventElapsedTime(&ms, E.tev[2 * i], E.tev[2 * i + 1]));
                const int cls = E.tmarks[i].first;
                c->t_ms[cls] += ms;
                c->t_launches[cls] += 1;
                c->t_bytes[cls] += E.tmarks[i].second * active / ncol;
            }
        if (c->timing) {
            active = 0;
            for (int i = 0; i < ncol; ++i) active += E.h_done[i] == 0;
        }
        if (debug_log() && (cyc < 30 || cyc % 50 == 0)) {
            SGN_CUDA(cudaMemcpy(E.h_resest, E.S.resest, ncol * sizeof(double), cudaMemcpyDeviceToHost));
            double mx = 0;
            for (int i = 0; i < ncol; ++i) mx = std::max(mx, E.h_resest[i]);
            fprintf(stderr, "[sgn cycle] %d resmax %.3e\n", cyc, mx);
        }
        if (*E.h_err) break;
        all_done = true;
        for (int i = 0; i < ncol; ++i) all_done = all_done && E.h_done[i];
        if (all_done) {
            ++cyc;
            break;
        }
    }
    }
finish:
    SGN_CUDA(cudaMemcpyAsync(E.h_resest, E.S.resest, ncol * sizeof(double), cudaMemcpyDeviceToHost, st));
    SGN_CUDA(cudaMemcpyAsync(E.h_kk, E.S.kk, ncol * sizeof(int), cudaMemcpyDeviceToHost, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    res->cycles = cyc;
    res->converged = all_done;
    res->err = *E.h_err;
    res->resmax = 0;
    for (int i = 0; i < ncol; ++i) res->resmax = std::max(res->resmax, E.h_resest[i]);
    if (res->err & 1) {
        set_error("a shifted Hessenberg system was singular (a shift lies on a Ritz value)");
        return SGN_ERR_BREAKDOWN;
    }
    if (res->err & 2) {
        set_error("non-finite value met in the Arnoldi process");
        return SGN_ERR_NONFINITE;
    }
    return SGN_OK;
}

int ensure_io(sgn_ctx* c, size_t bytes) {
    if (c->io.p && c->io.bytes >= bytes) return SGN_OK;
    SGN_CUDA(cudaStreamSynchronize(c->work));
    return dev_alloc(c, c->io, bytes);
}

int fill_shift_tables(sgn_ctx* c, Engine& E, const double* sig_cols, const double* om_cols,
                      const double* sig_im_cols = nullptr) {
    const size_t bytes = sizeof(double) * E.ncol * E.s;
    SGN_CUDA(cudaMemcpyAsync(E.sigma_dev, sig_cols, bytes, cudaMemcpyHostToDevice, c->work));
    SGN_CUDA(cudaMemcpyAsync(E.omega_dev, om_cols, bytes, cudaMemcpyHostToDevice, c->work));
    if (sig_im_cols)
        SGN_CUDA(cudaMemcpyAsync(E.sigma_im_dev, sig_im_cols, bytes, cudaMemcpyHostToDevice, c->work));
    else
        SGN_CUDA(cudaMemsetAsync(E.sigma_im_dev, 0, bytes, c->work));
    return SGN_OK;
}

}  // namespace

namespace {

// Mixed form.  Phase 1: Algorithm 1 with the FP32 stencil and FP32 Krylov
// basis (inner products, norms, Hessenberg matrix, shifted solves, rho and the
// projection coefficients in FP64), accumulating every shifted iterate x_i in
// FP64.  Phase 2 (iterative refinement, not part of the paper): the true
// residual r_i = b~ - (A^2 - sigma_i) x_i of every shifted system is formed in
// FP64; systems whose relative residual exceeds the tolerance get a correction
// d_i from restarted FOM on (A^2 - sigma_i) d = (I - P) r_i, again FP32 basis
// with FP64 scalars, batched one system per column; x_i += d_i.  Rounds repeat
// until every true residual meets the tolerance that stops the FP64 form.
constexpr size_t kRefineBudgetBytes = size_t(48) << 30;

int solve_mixed(sgn_ctx* c, const double2* b, double2* x, double2* x_shift, int ncol, bool adjoint, bool no_a,
                sgn_report* rep) {
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    const int s = (int)c->sigma.size();
    const int k = c->k;
    const int m = c->m;
    Engine* E = nullptr;
    SGN_CHECK(get_engine(c, ncol, k, s, SGN_PREC_MIXED, &E));
    // refinement batch: one shifted system per column, bounded by memory.  The
    // corrections only have to gain a factor tol / (FP32 floor ~1e-6) and most of
    // them converge in a few steps, so they restart sooner than the multishift
    // phase: a cycle of the engine always runs all its k_refine steps.
    const int k1 = c->k_refine > 0 ? c->k_refine : std::min(k, 16);
    const size_t per_col = (size_t)(k1 + 4) * n * sizeof(float2) + (size_t)n * sizeof(double2);
    size_t bmax = c->refine_batch > 0 ? (size_t)c->refine_batch : (size_t)10 * ncol;
    int B = (int)std::min<size_t>({(size_t)s * ncol, bmax, std::max<size_t>(1, kRefineBudgetBytes / per_col)});
    Engine* E1 = nullptr;
    SGN_CHECK(get_engine(c, B, k1, 1, SGN_PREC_MIXED, &E1));

    // io: xs (s ncol) | r0, bt, xP, t, u (ncol each) | d (B) | omega table | FP64 partials
    const size_t field = (size_t)n * sizeof(double2);
    const int nblk64 = reduce_blocks<double2>(n);
    const int rs64 = ((std::max(m, s) + 2) + 7) & ~7;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    size_t o_xs = take(field * ncol * s);
    size_t o_r0 = take(field * ncol), o_bt = take(field * ncol), o_xp = take(field * ncol);
    size_t o_t = take(field * ncol), o_u = take(field * ncol);
    size_t o_d = take(field * B);
    size_t o_rs = take(field * ncol * s);
    const int ncmax = std::max({ncol, B, s * ncol});
    size_t o_om = take(sizeof(double2) * ncol * rs64);
    size_t o_red = take(sizeof(double2) * ncmax * rs64);
    size_t o_part = take(sizeof(double2) * (size_t)ncmax * rs64 * nblk64);
    size_t o_flags = take(sizeof(int) * 2 * ncmax);
    size_t o_roff = take(sizeof(long long) * B), o_rsig = take(sizeof(double) * B);
    SGN_CHECK(ensure_io(c, off));
    char* io = reinterpret_cast<char*>(c->io.p);
    double2* xs = reinterpret_cast<double2*>(io + o_xs);
    double2* r0 = reinterpret_cast<double2*>(io + o_r0);
    double2* bt = reinterpret_cast<double2*>(io + o_bt);
    double2* xP = reinterpret_cast<double2*>(io + o_xp);
    double2* t64 = reinterpret_cast<double2*>(io + o_t);
    double2* u64 = reinterpret_cast<double2*>(io + o_u);
    double2* d = reinterpret_cast<double2*>(io + o_d);
    double2* rsd = reinterpret_cast<double2*>(io + o_rs);  // true residuals r_i, [i][col][n]
    double2* omtab = reinterpret_cast<double2*>(io + o_om);
    long long* roff_dev = reinterpret_cast<long long*>(io + o_roff);
    double* rsig_dev = reinterpret_cast<double*>(io + o_rsig);
    // FP64 reductions use their own partials and state (the FP32 engines size theirs for float packs)
    DevState S64{};
    S64.red = reinterpret_cast<double2*>(io + o_red);
    S64.skip = reinterpret_cast<int*>(io + o_flags);
    S64.done = S64.skip + ncmax;
    S64.rstride = rs64;
    const Reduce rd64{reinterpret_cast<double2*>(io + o_part), nblk64, rs64};
    SGN_CUDA(cudaMemsetAsync(S64.skip, 0, sizeof(int) * 2 * ncmax, st));

    std::vector<double> sig_cols((size_t)ncol * s), om_cols((size_t)ncol * s);
    std::vector<double2> omh((size_t)ncol * rs64, make_double2(0, 0));
    for (int col = 0; col < ncol; ++col)
        for (int i = 0; i < s; ++i) {
            sig_cols[(size_t)col * s + i] = c->sigma[i];
            om_cols[(size_t)col * s + i] = c->omega[i];
            omh[(size_t)col * rs64 + i] = make_double2(c->omega[i], 0);
        }
    SGN_CHECK(fill_shift_tables(c, *E, sig_cols.data(), om_cols.data()));
    SGN_CUDA(cudaMemcpyAsync(omtab, omh.data(), sizeof(double2) * omh.size(), cudaMemcpyHostToDevice, st));

    const double2* Lb = reinterpret_cast<const double2*>(adjoint ? c->R64.p : c->L64.p);
    const double2* Rb = reinterpret_cast<const double2*>(adjoint ? c->L64.p : c->R64.p);
    const float2* Lb32 = reinterpret_cast<const float2*>(adjoint ? c->R32.p : c->L32.p);
    const float2* Rb32 = reinterpret_cast<const float2*>(adjoint ? c->L32.p : c->R32.p);
    const double2* lam = reinterpret_cast<const double2*>(adjoint ? c->lamc_dev.p : c->lam_dev.p);
    const Basis<double2> LB{Lb, n, 0}, RB{Rb, n, 0};

    SGN_CUDA(cudaMemsetAsync(xs, 0, field * ncol * s, st));
    SGN_CUDA(cudaMemsetAsync(xP, 0, field * ncol, st));
    const double2* rstart = b;
    if (m > 0) {
        SGN_CUDA(mdot<double2>(LB, m, b, n, n, ncol, rd64, 0, nullptr, st));
        SGN_CUDA(reduce(rd64, m, ncol, RM_SIGNED, 0, S64, lam, st));
        SGN_CUDA(update_x<double2>(RB, m, S64.red, rs64, xP, n, n, ncol, nullptr, nullptr, st));
        SGN_CUDA(reduce(rd64, m, ncol, RM_STORE, 0, S64, nullptr, st));
        SGN_CUDA(maxpy_scale<double2>(RB, m, S64.red, rs64, b, n, r0, n, nullptr, n, ncol, nullptr, st));
        rstart = r0;
    }
    if (no_a)
        SGN_CUDA(cudaMemcpyAsync(bt, rstart, field * ncol, cudaMemcpyDeviceToDevice, st));
    else
        SGN_CUDA(apply_hw64(c, bt, rstart, ncol, adjoint, nullptr, st));  // b~ in FP64
    SGN_CUDA(convert_f64_to_f32(bt, reinterpret_cast<float2*>(E->V), (int64_t)ncol * n, st));
    const int p32 = stencil_prec32(c);
    SGN_CHECK(tune_stencil(c, p32, ncol, E->V, E->t));
    SGN_CHECK(tune_stencil(c, p32, B, E1->V, E1->t));
    SGN_CHECK(tune_stencil(c, 0, ncol, bt, t64));

    CycleArgs a;
    a.adjoint = adjoint;
    a.L = Lb32;
    a.R = Rb32;
    a.m = m;
    a.project = c->project;
    a.xs = xs;
    a.xs_shift = (int64_t)ncol * n;
    a.xs_col = n;
    const double tol_inner = std::max(c->tol, 1e-6);
    RunResult rr;
    int status = run_engine<float2>(c, *E, a, tol_inner, c->max_cycles, &rr);
    if (debug_log())
        fprintf(stderr, "[sgn mixed] multishift phase: status %d cycles %d converged %d resmax %.3e err %d\n", status,
                rr.cycles, rr.converged, rr.resmax, rr.err);
    if (status != SGN_OK) return status;
    const int ms_cycles = rr.cycles;
    int ref_rounds = 0, ref_cycles = 0;
    double worst = 0;

    // ||b~|| per column (FP64)
    std::vector<double> bnorm(ncol);
    {
        SGN_CUDA(mdot<double2>(Basis<double2>{bt, 0, n}, 0, bt, n, n, ncol, rd64, 1, nullptr, st));
        SGN_CUDA(reduce(rd64, 1, ncol, RM_STORE, 0, S64, nullptr, st));
        std::vector<double2> h((size_t)ncol * rs64);
        SGN_CUDA(cudaMemcpyAsync(h.data(), S64.red, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        for (int col = 0; col < ncol; ++col) bnorm[col] = std::sqrt(h[(size_t)col * rs64].x);
    }

    CycleArgs a1;
    a1.adjoint = adjoint;
    a1.L = Lb32;
    a1.R = Rb32;
    a1.m = m;
    a1.project = c->project;
    a1.xs = d;
    a1.xs_shift = (int64_t)B * n;
    a1.xs_col = n;
    // Correction solves by restarted FOM (Galerkin, like the multishift phase); a batch whose
    // FOM does not converge within kFomCap cycles, or meets a non-finite value, is solved again
    // from the same residuals with minimal-residual (GMRES) restarts.  Restarted FOM on a single
    // strongly non-normal shifted system can diverge (at mu = 1 its residual grew without bound
    // over 1,800 cycles); GMRES cannot.  GMRES corrections leave residuals along unrelated
    // directions, whose errors add up less favourably: the retry aims at a third of the target
    // (on the 10^4 workload at tol 1e-8, GMRES corrections gave a relative error of x of 1.4e-8
    // at the target and 4.7e-9 at a third of it; FOM corrections 2.9e-9 at the target).
    constexpr int kFomCap = 300;
    const double rtol = c->tol;
    const int max_rounds = 8;
    std::vector<double> sig1(B), om1(B, 1.0);
    const int nall = s * ncol;  // every (shift, column) pair as one column of [i][col][n]
    std::vector<double2> hall((size_t)nall * rs64);
    std::vector<long long> roff(B);
    std::vector<double> rsig(B);
    for (int round = 0; round <= max_rounds; ++round) {
        // true residuals r_i = b~ - (A^2 - sigma_i) x_i of every shifted system: from
        // scratch in refinement round 0, assembled in FP64; later rounds carry them along with
        // the corrections (r_i -= R c_i with x_i += R (Lambda^2 - sigma_i)^{-1} c_i,
        // r_i -= (A^2 - sigma_i) d_i with x_i += d_i), where FP32 products of the small d_i are
        // exact to ~1e-7 ||r_i||.
        // Round 0 forms A^2 x_i in float-float arithmetic on the FP32 units (stencil_ff.cu; ~1e-13
        // of the FP64 stencil, which GB300 runs at 1/64 of the FP32 rate); the (hi, lo) pairs of
        // x_i and A x_i live in the space of t64 and u64 (4 ncol complex64 fields = 2 ncol
        // complex128 fields).
        if (round == 0) {
            const size_t nf = (size_t)ncol * n;
            float2* xh = reinterpret_cast<float2*>(t64);
            float2* xl = xh + nf;
            float2* th = reinterpret_cast<float2*>(u64);
            float2* tl = th + nf;
            const StencilParams pf = stencil_params(c, adjoint);
            const float4* Uf = reinterpret_cast<const float4*>(c->Uff.p);
            for (int i = 0; i < s; ++i) {
                double2* xi = xs + (size_t)i * nf;
                SGN_CUDA(split_ff(xi, xh, xl, (int64_t)nf, st));
                SGN_CUDA(launch_hw_ff(th, tl, xh, xl, Uf, ncol, pf, st));
                SGN_CUDA(launch_hw_ff(xh, xl, th, tl, Uf, ncol, pf, st));
                SGN_CUDA(residual_ff(rsd + (size_t)i * nf, bt, xh, xl, c->sigma[i], xi, (int64_t)nf, st));
            }
        }
        SGN_CUDA(mdot<double2>(Basis<double2>{rsd, 0, n}, 0, rsd, n, n, nall, rd64, 1, nullptr, st));
        SGN_CUDA(reduce(rd64, 1, nall, RM_STORE, 0, S64, nullptr, st));
        SGN_CUDA(cudaMemcpyAsync(hall.data(), S64.red, sizeof(double2) * hall.size(), cudaMemcpyDeviceToHost, st));
        SGN_CUDA(cudaStreamSynchronize(st));
        std::vector<std::pair<int, int>> todo;  // (shift, column)
        std::vector<double> todo_rel;           // its relative true residual
        worst = 0;
        for (int i = 0; i < s; ++i)
            for (int col = 0; col < ncol; ++col) {
                const double r2 = hall[((size_t)i * ncol + col) * rs64].x;
                const double rel = bnorm[col] > 0 ? std::sqrt(r2) / bnorm[col] : 0.0;
                if (!std::isfinite(rel)) {
                    set_error("non-finite true residual in refinement");
                    return SGN_ERR_NONFINITE;
                }
                worst = std::max(worst, rel);
                if (rel > rtol) {
                    todo.emplace_back(i, col);
                    todo_rel.push_back(rel);
                }
            }
        if (debug_log())
            fprintf(stderr, "[sgn mixed] round %d: worst true residual %.3e, %zu of %d systems above tol\n", round,
                    worst, todo.size(), nall);
        if (todo.empty() || round == max_rounds) break;
        ++ref_rounds;
        if (m > 0) {
            // the range(P) part of each residual is solved exactly in the eigenbasis,
            // (A^2 - sigma)^{-1} R = R (Lambda^2 - sigma)^{-1}:  x_i += R (Lambda^2 - sigma_i)^{-1} L^dag r_i,
            // and the Krylov corrections work on (I - P) r_i.  One launch each for all pairs,
            // with the FP32 copies of L and R read once per tile of columns (tsmm.cu).
            SGN_CUDA(tsmm_tn<float2>(Lb32, n, m, rsd, n, nall, n, rd64, st));
            SGN_CUDA(reduce(rd64, m, nall, RM_STORE, 0, S64, nullptr, st));
            SGN_CUDA(tsmm_nn<float2>(Rb32, n, m, S64.red, rs64, rsd, n, nall, n, -1.0, st));
            SGN_CUDA(cudaMemcpyAsync(hall.data(), S64.red, sizeof(double2) * hall.size(), cudaMemcpyDeviceToHost, st));
            SGN_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i < s; ++i)
                for (int col = 0; col < ncol; ++col)
                    for (int l = 0; l < m; ++l) {
                        double2& v = hall[((size_t)i * ncol + col) * rs64 + l];
                        const std::complex<double> lj = adjoint ? std::conj(c->lam[l]) : c->lam[l];
                        const std::complex<double> q = std::complex<double>(v.x, v.y) / (lj * lj - c->sigma[i]);
                        v = make_double2(q.real(), q.imag());
                    }
            SGN_CUDA(cudaMemcpyAsync(S64.red, hall.data(), sizeof(double2) * hall.size(), cudaMemcpyHostToDevice, st));
            SGN_CUDA(tsmm_nn<float2>(Rb32, n, m, S64.red, rs64, xs, n, nall, n, 1.0, st));
            SGN_CUDA(cudaStreamSynchronize(st));
        }
        // correction solves, B systems at a time, one system per column
        for (size_t t0 = 0; t0 < todo.size(); t0 += B) {
            const int nb = (int)std::min<size_t>(B, todo.size() - t0);
            float2* V0 = reinterpret_cast<float2*>(E1->V);
            for (int j = 0; j < B; ++j) sig1[j] = j < nb ? c->sigma[todo[t0 + j].first] : c->sigma[0];
            SGN_CHECK(fill_shift_tables(c, *E1, sig1.data(), om1.data()));
            // the correction needs to reduce the worst residual of the batch to a third
            // of the tolerance, not further (FP32 bases reach about 1e-6 at best)
            double brel = 0;
            for (int j = 0; j < nb; ++j) brel = std::max(brel, todo_rel[t0 + j]);
            int st1 = SGN_OK;
            RunResult r1;
            for (int attempt = 0; attempt < 2; ++attempt) {
                a1.gmres = attempt == 1;
                SGN_CUDA(cudaMemsetAsync(V0, 0, sizeof(float2) * (size_t)B * n, st));
                for (int j = 0; j < nb; ++j) {
                    const int i = todo[t0 + j].first, col = todo[t0 + j].second;
                    SGN_CUDA(convert_f64_to_f32(rsd + ((size_t)i * ncol + col) * n, V0 + (size_t)j * n, n, st));
                }
                SGN_CUDA(cudaMemsetAsync(d, 0, field * B, st));
                const double inner = std::min(0.1, std::max(1e-5, rtol / ((a1.gmres ? 9.0 : 3.0) * brel)));
                st1 = run_engine<float2>(c, *E1, a1, inner, a1.gmres ? c->max_cycles : std::min(c->max_cycles, kFomCap),
                                         &r1);
                if (debug_log())
                    fprintf(stderr,
                            "[sgn mixed]   batch at %zu (%d systems, %s): inner tol %.1e status %d cycles %d "
                            "resmax %.3e\n",
                            t0, nb, a1.gmres ? "GMRES" : "FOM", inner, st1, r1.cycles, r1.resmax);
                ref_cycles += r1.cycles;
                const bool fom_failed = !a1.gmres && (st1 == SGN_ERR_NONFINITE || st1 == SGN_ERR_BREAKDOWN ||
                                                      (st1 == SGN_OK && !r1.converged));
                if (!fom_failed) break;
                SGN_CUDA(cudaMemsetAsync(E1->S.err, 0, sizeof(int), st));
            }
            if (st1 != SGN_OK) return st1;
            // r_i -= (A^2 - sigma_i) d_i:  A^2 d in FP32 on the engine's scratch fields
            {
                float2* w32 = reinterpret_cast<float2*>(E1->w);
                float2* t32 = reinterpret_cast<float2*>(E1->t);
                SGN_CUDA(convert_f64_to_f32(d, w32, (int64_t)nb * n, st));
                // FP32 links even when the solves run on BF16 ones: the carried residual
                // must see the true operator, not the one the corrections were solved with
                SGN_CUDA(apply_hw32(c, t32, w32, nb, adjoint, nullptr, st, true));
                SGN_CUDA(apply_hw32(c, w32, t32, nb, adjoint, nullptr, st, true));
                for (int j = 0; j < nb; ++j) {
                    roff[j] = (long long)((size_t)todo[t0 + j].first * ncol + todo[t0 + j].second) * n;
                    rsig[j] = c->sigma[todo[t0 + j].first];
                }
                SGN_CUDA(cudaMemcpyAsync(roff_dev, roff.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice, st));
                SGN_CUDA(cudaMemcpyAsync(rsig_dev, rsig.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
                SGN_CUDA(correct_residuals(rsd, roff_dev, rsig_dev, w32, d, n, nb, st));
            }
            for (int j = 0; j < nb; ++j) {
                const int i = todo[t0 + j].first, col = todo[t0 + j].second;
                double2* xi = xs + ((size_t)i * ncol + col) * n;
                SGN_CUDA(axpby3<double2>(xi, 1.0, xi, 1.0, d + (size_t)j * n, 0.0, nullptr, n, st));
            }
        }
    }
    // x = x_P + sum_i omega_i x_i
    SGN_CUDA(cudaMemcpyAsync(x, xP, field * ncol, cudaMemcpyDeviceToDevice, st));
    SGN_CUDA(update_x<double2>(Basis<double2>{xs, (int64_t)ncol * n, n}, s, omtab, rs64, x, n, n, ncol, nullptr,
                               nullptr, st));
    if (x_shift) SGN_CUDA(cudaMemcpyAsync(x_shift, xs, field * ncol * s, cudaMemcpyDeviceToDevice, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    if (worst > rtol) {
        status = SGN_ERR_NOT_CONVERGED;
        set_error("mixed form: refinement did not bring every true residual below the tolerance");
    }
    if (rep) {
        rep->status = status;
        rep->cycles = ms_cycles;
        rep->matvecs = 1 + 2 * k * ms_cycles;
        rep->refine_rounds = ref_rounds;
        rep->refine_cycles = ref_cycles;
        rep->res_est = rr.resmax;
        rep->err_est = worst;
        rep->breakdown = 0;
    }
    return status;
}

}  // namespace

// x = x_P + sum_i omega_i x_i on ncol device fields (FP64).  See sgn_apply.
int solve(sgn_ctx* c, const double2* b, double2* x, double2* x_shift, int ncol, bool adjoint, bool no_a,
          sgn_report* rep, const std::vector<std::complex<double>>* cshift) {
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    // Shifted systems and weights: cshift (complex shifts, unit weights); the split form
    // t / (t^2 - sigma) = 1/2 [(t - a)^{-1} + (t + a)^{-1}], a = sqrt(sigma): 2s systems in A
    // itself with weights omega/2 and no A on the right-hand side; else eq. (6.2)'s s
    // systems in A^2.
    const bool split = !cshift && c->form == SGN_FORM_A;
    std::vector<std::complex<double>> sh;
    std::vector<double> wt;
    if (cshift) {
        sh = *cshift;
        wt.assign(sh.size(), 1.0);
    } else if (split) {
        for (size_t i = 0; i < c->sigma.size(); ++i) {
            const std::complex<double> a = std::sqrt(std::complex<double>(c->sigma[i], 0.0));
            sh.push_back(a);
            sh.push_back(-a);
            wt.push_back(0.5 * c->omega[i]);
            wt.push_back(0.5 * c->omega[i]);
        }
    } else {
        for (size_t i = 0; i < c->sigma.size(); ++i) {
            sh.push_back(c->sigma[i]);
            wt.push_back(c->omega[i]);
        }
    }
    const int s = (int)sh.size();
    const int k = c->k;
    const int m = c->m;
    if (split && (c->precision == SGN_PREC_MIXED || x_shift)) {
        set_error("solve: the split form (Krylov space of A) runs in the FP64 form, without per-shift output");
        return SGN_ERR_STATE;
    }
    if (split) no_a = true;
    // GMRES-LR: restarted multishift GMRES; the seed (minimal residual) is the shift of
    // smallest modulus, the slowest to converge, moved to position 0
    const bool gm = !cshift && c->method == SGN_METHOD_GMRES;
    if (gm && (split || c->precision == SGN_PREC_MIXED)) {
        set_error("solve: GMRES-LR runs in the FP64 form of the A^2 formulation");
        return SGN_ERR_STATE;
    }
    int seed = 0;
    if (gm) {
        for (int i = 1; i < (int)sh.size(); ++i)
            if (std::abs(sh[i]) < std::abs(sh[seed])) seed = i;
        std::swap(sh[0], sh[seed]);
        std::swap(wt[0], wt[seed]);
    }
    if (c->precision == SGN_PREC_MIXED && !cshift) return solve_mixed(c, b, x, x_shift, ncol, adjoint, no_a, rep);
    if (s < 1) {
        set_error("solve: no shifts");
        return SGN_ERR_ARG;
    }
    Engine* E = nullptr;
    SGN_CHECK(get_engine(c, ncol, k, s, SGN_PREC_FP64, &E));
    // io: xacc (ncol n) | r0 (ncol n) | xs (s ncol n, optional)
    const size_t field = (size_t)n * sizeof(double2);
    const size_t f_cols = align256(field * ncol);
    const size_t need = 2 * f_cols + (x_shift ? align256(field * ncol * s) : 0);
    SGN_CHECK(ensure_io(c, need));
    char* io = reinterpret_cast<char*>(c->io.p);
    double2* xacc = reinterpret_cast<double2*>(io);
    double2* r0 = reinterpret_cast<double2*>(io + f_cols);
    double2* xs = x_shift ? reinterpret_cast<double2*>(io + 2 * f_cols) : nullptr;

    std::vector<double> sig_cols((size_t)ncol * s), om_cols((size_t)ncol * s), sim_cols((size_t)ncol * s, 0.0);
    for (int col = 0; col < ncol; ++col)
        for (int i = 0; i < s; ++i) {
            sig_cols[(size_t)col * s + i] = sh[i].real();
            sim_cols[(size_t)col * s + i] = sh[i].imag();
            om_cols[(size_t)col * s + i] = wt[i];
        }
    SGN_CHECK(fill_shift_tables(c, *E, sig_cols.data(), om_cols.data(), sim_cols.data()));

    const double2* Lb = reinterpret_cast<const double2*>(adjoint ? c->R64.p : c->L64.p);
    const double2* Rb = reinterpret_cast<const double2*>(adjoint ? c->L64.p : c->R64.p);
    const double2* lam = reinterpret_cast<const double2*>(adjoint ? c->lamc_dev.p : c->lam_dev.p);
    const Reduce rd{E->partial, E->nblk, E->rstride};
    SGN_CUDA(cudaMemsetAsync(E->S.done, 0, ncol * sizeof(int), st));
    SGN_CUDA(cudaMemsetAsync(E->S.skip, 0, ncol * sizeof(int), st));
    SGN_CUDA(cudaMemsetAsync(xacc, 0, field * ncol, st));
    if (xs) SGN_CUDA(cudaMemsetAsync(xs, 0, field * ncol * s, st));
    const double2* rstart = b;
    if (m > 0) {
        // x = x_P = R f(Lambda) L^dag b (eq. (4.3)); r = (I - P) b (eq. (4.2))
        const Basis<double2> LB{Lb, n, 0}, RB{Rb, n, 0};
        SGN_CUDA(mdot<double2>(LB, m, b, n, n, ncol, rd, 0, nullptr, st));
        SGN_CUDA(reduce(rd, m, ncol, RM_SIGNED, 0, E->S, lam, st));
        SGN_CUDA(update_x<double2>(RB, m, E->S.red, E->rstride, xacc, n, n, ncol, nullptr, nullptr, st));
        SGN_CUDA(reduce(rd, m, ncol, RM_STORE, 0, E->S, nullptr, st));
        SGN_CUDA(maxpy_scale<double2>(RB, m, E->S.red, E->rstride, b, n, r0, n, nullptr, n, ncol, nullptr, st));
        rstart = r0;
    }
    // b~ = A (I - P) b is the first restart vector (A^2 reading of eq. (6.2))
    if (no_a)
        SGN_CUDA(cudaMemcpyAsync(E->V, rstart, field * ncol, cudaMemcpyDeviceToDevice, st));
    else
        SGN_CUDA(apply_hw64(c, reinterpret_cast<double2*>(E->V), rstart, ncol, adjoint, nullptr, st));

    SGN_CHECK(tune_stencil(c, 0, ncol, E->V, E->t));
    CycleArgs a;
    a.adjoint = adjoint;
    a.L = Lb;
    a.R = Rb;
    a.m = m;
    a.project = c->project;
    a.xacc = xacc;
    a.xsr = n;
    a.xs = xs;
    a.xs_shift = (int64_t)ncol * n;
    a.xs_col = n;
    a.op_a = split;
    a.gmres = gm;
    RunResult rr;
    int status = run_engine<double2>(c, *E, a, c->tol, c->max_cycles, &rr);
    if (!cshift) c->last_fp64 = E;
    if (status == SGN_OK) {
        SGN_CUDA(cudaMemcpyAsync(x, xacc, field * ncol, cudaMemcpyDeviceToDevice, st));
        if (x_shift && seed == 0) SGN_CUDA(cudaMemcpyAsync(x_shift, xs, field * ncol * s, cudaMemcpyDeviceToDevice, st));
        if (x_shift && seed != 0) {  // undo the seed's move: engine slots 0 and seed trade places
            const size_t blk = field * ncol;
            char* dst = reinterpret_cast<char*>(x_shift);
            const char* src = reinterpret_cast<const char*>(xs);
            SGN_CUDA(cudaMemcpyAsync(dst, src, blk * s, cudaMemcpyDeviceToDevice, st));
            SGN_CUDA(cudaMemcpyAsync(dst, src + blk * seed, blk, cudaMemcpyDeviceToDevice, st));
            SGN_CUDA(cudaMemcpyAsync(dst + blk * seed, src, blk, cudaMemcpyDeviceToDevice, st));
        }
        if (!rr.converged) {
            status = SGN_ERR_NOT_CONVERGED;
            set_error("max_cycles reached before every shifted system met the tolerance");
        }
    }
    if (rep) {
        rep->status = status;
        rep->cycles = rr.cycles;
        rep->matvecs = split ? k * rr.cycles : 1 + 2 * k * rr.cycles;
        rep->refine_rounds = 0;
        rep->refine_cycles = 0;
        rep->res_est = rr.resmax;
        rep->err_est = 0;
        int bd = 0;
        for (int i = 0; i < ncol; ++i) bd |= E->h_kk[i] < k;
        rep->breakdown = bd;
    }
    return status;
}

// (A^2 - shift_col)^{-1} (I - P) rhs_col for ncol columns, one complex shift each (A^dag
// with adjoint), by restarted GMRES in the FP64 engine: minimal-residual restarts, the
// deflation projection after every cycle, no A applied to the right-hand side.  Shifts
// inside the field of values of A^2 (where FOM's H_k - shift can be singular) are fine.
int solve_columns_gmres(sgn_ctx* c, const double2* rhs, int ncol, const std::vector<std::complex<double>>& shift,
                        bool adjoint, double2* out, const double2* Rp, const double2* Lp, int mp) {
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    const int k = c->k;
    const int m = mp;  // projected pairs: Rp, Lp (n x mp, biorthonormal), null for none
    if ((int)shift.size() != ncol || ncol < 1 || (m > 0 && (!Rp || !Lp))) {
        set_error("solve_columns_gmres: one shift per column");
        return SGN_ERR_ARG;
    }
    // batches bounded by the engine's memory (k + 4 fields per column)
    const size_t per_col = (size_t)(k + 4) * n * sizeof(double2);
    const int bmax = (int)std::max<size_t>(1, std::min<size_t>(ncol, kRefineBudgetBytes / 2 / per_col));
    if (ncol > bmax) {
        for (int c0 = 0; c0 < ncol; c0 += bmax) {
            const int nb = std::min(bmax, ncol - c0);
            std::vector<std::complex<double>> sub(shift.begin() + c0, shift.begin() + c0 + nb);
            SGN_CHECK(solve_columns_gmres(c, rhs + (size_t)c0 * n, nb, sub, adjoint, out + (size_t)c0 * n, Rp, Lp, mp));
        }
        return SGN_OK;
    }
    // the engine key includes c->m; the projection count here is mp
    const int m_saved = c->m;
    c->m = mp;
    Engine* E = nullptr;
    const int ge = get_engine(c, ncol, k, 1, SGN_PREC_FP64, &E);
    c->m = m_saved;
    SGN_CHECK(ge);
    const size_t field = (size_t)n * sizeof(double2);
    std::vector<double> sig(ncol), sim(ncol), om(ncol, 1.0);
    for (int col = 0; col < ncol; ++col) {
        sig[col] = shift[col].real();
        sim[col] = shift[col].imag();
    }
    SGN_CHECK(fill_shift_tables(c, *E, sig.data(), om.data(), sim.data()));
    const double2* Lb = adjoint ? Rp : Lp;
    const double2* Rb = adjoint ? Lp : Rp;
    SGN_CUDA(cudaMemsetAsync(E->S.done, 0, ncol * sizeof(int), st));
    SGN_CUDA(cudaMemsetAsync(E->S.skip, 0, ncol * sizeof(int), st));
    SGN_CUDA(cudaMemsetAsync(out, 0, field * ncol, st));
    double2* V0 = reinterpret_cast<double2*>(E->V);
    SGN_CUDA(cudaMemcpyAsync(V0, rhs, field * ncol, cudaMemcpyDeviceToDevice, st));
    if (m > 0) {  // r = (I - P) rhs
        const Reduce rd{E->partial, E->nblk, E->rstride};
        const Basis<double2> LB{Lb, n, 0}, RB{Rb, n, 0};
        SGN_CUDA(mdot<double2>(LB, m, V0, n, n, ncol, rd, 0, nullptr, st));
        SGN_CUDA(reduce(rd, m, ncol, RM_STORE, 0, E->S, nullptr, st));
        SGN_CUDA(maxpy_scale<double2>(RB, m, E->S.red, E->rstride, V0, n, V0, n, nullptr, n, ncol, nullptr, st));
    }
    SGN_CHECK(tune_stencil(c, 0, ncol, E->V, E->t));
    CycleArgs a;
    a.adjoint = adjoint;
    a.L = Lb;
    a.R = Rb;
    a.m = m;
    a.project = 1;
    a.xs = out;
    a.xs_shift = (int64_t)ncol * n;
    a.xs_col = n;
    a.gmres = true;
    RunResult rr;
    int status = run_engine<double2>(c, *E, a, c->tol, c->max_cycles, &rr);
    if (status == SGN_OK && !rr.converged) {
        status = SGN_ERR_NOT_CONVERGED;
        set_error("solve_columns_gmres: max_cycles reached before every system met the tolerance");
    }
    return status;
}

int field_dots(sgn_ctx* c, const double2* a, const double2* b, int ncol, std::vector<std::complex<double>>& out) {
    cudaStream_t st = c->work;
    const int64_t n = c->n;
    const int nblk = reduce_blocks<double2>(n);
    const int rs = 8;
    DevBuf buf;
    const size_t pbytes = align256(sizeof(double2) * (size_t)ncol * rs * nblk);
    SGN_CHECK(dev_alloc(c, buf, pbytes + align256(sizeof(double2) * ncol * rs) + align256(sizeof(int) * 2 * ncol)));
    char* p = reinterpret_cast<char*>(buf.p);
    DevState S{};
    S.red = reinterpret_cast<double2*>(p + pbytes);
    S.skip = reinterpret_cast<int*>(p + pbytes + align256(sizeof(double2) * ncol * rs));
    S.done = S.skip + ncol;
    S.rstride = rs;
    SGN_CUDA(cudaMemsetAsync(S.skip, 0, sizeof(int) * 2 * ncol, st));
    const Reduce rd{reinterpret_cast<double2*>(p), nblk, rs};
    SGN_CUDA(mdot<double2>(Basis<double2>{a, 0, n}, 1, b, n, n, ncol, rd, 0, nullptr, st));
    SGN_CUDA(reduce(rd, 1, ncol, RM_STORE, 0, S, nullptr, st));
    std::vector<double2> h((size_t)ncol * rs);
    SGN_CUDA(cudaMemcpyAsync(h.data(), S.red, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
    SGN_CUDA(cudaStreamSynchronize(st));
    dev_free(c, buf);
    out.resize(ncol);
    for (int i = 0; i < ncol; ++i) out[i] = {h[(size_t)i * rs].x, h[(size_t)i * rs].y};
    return SGN_OK;
}

}  // namespace sgn
