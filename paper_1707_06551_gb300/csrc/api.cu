// C interface (include/sphere_bie.h): context lifetime, operator assembly
// (Sec. 4.3), GMRES on the device and the mobility (Eq. 5.8) and resistance
// (Eq. 5.19) drivers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "common.h"

using namespace sbie;

static std::string g_last_error = "no error";

void sbie::set_last_error(const std::string& msg) { g_last_error = msg; }

#define CK(expr)                                                            \
    do {                                                                    \
        cudaError_t e__ = (expr);                                           \
        if (e__ != cudaSuccess) {                                           \
            c->err = std::string(#expr) + ": " + cudaGetErrorString(e__);   \
            return SBIE_ERR_CUDA;                                           \
        }                                                                   \
    } while (0)

#define CKS(expr)                                   \
    do {                                            \
        sbie_status s__ = (expr);                   \
        if (s__ != SBIE_OK) return s__;             \
    } while (0)

namespace {

sbie_status fail(sbie_ctx* c, sbie_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_last_error = msg;
    return s;
}

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1));
}

void free_all(sbie_ctx* c) {
    void* ptrs[] = {c->d_c, c->d_a, c->d_x, c->d_xhi, c->d_xlo, c->d_nrm, c->d_nrm64, c->d_sph, c->d_near_ptr,
                    c->d_near_idx, c->d_tab, c->d_coef, c->d_chan, c->d_chanf, c->d_mom, c->d_part, c->d_src64,
                    c->d_srcf, c->d_in, c->d_out, c->d_tmp, c->d_tmp2, c->d_small, c->d_red, c->d_V, c->d_xsol,
                    c->d_rhs, c->d_res};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->h_red) cudaFreeHost(c->h_red);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (auto& v : c->prof_events)
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Far-field tilings found by sphere_bie_autotune, by (n, p, SM count, op, f32).
std::map<std::tuple<int, int, int, int, int>, FarTune> g_tune_cache;
std::mutex g_tune_mu;

void choose_tuning(sbie_ctx* c) {
    // Default tiling: targets per thread / threads per CTA with the fewest idle
    // target slots per sphere, then enough source splits for several CTAs per SM.
    auto pick = [&](bool f32) {
        FarTune best{128, f32 ? 2 : 1, 1, 256};
        double best_waste = 1e30;
        const int tpts[3] = {1, 2, 4};
        for (int tpt : tpts) {
            if (f32 && tpt == 1) continue;  // the FP32 kernel holds targets in pairs
            for (int th = 64; th <= 256; th += 32) {
                int slots = th * tpt;
                int chunks = (c->npn + slots - 1) / slots;
                double waste = (double)(chunks * slots - c->npn) / c->npn;
                double pref = f32 ? (tpt == 2 ? 0.0 : 0.03) : (tpt == 1 ? 0.0 : 0.05);
                pref += th == 128 ? 0.0 : 0.001;
                double score = waste + pref;
                if (score < best_waste - 1e-12) {
                    best_waste = score;
                    best = FarTune{th, tpt, 1, f32 ? 256 : 128};
                }
            }
        }
        int chunks = (c->npn + best.threads * best.tpt - 1) / (best.threads * best.tpt);
        long long ctas = (long long)c->n * chunks;
        long long want = (long long)c->sm_count * (f32 ? 12 : 4);
        int split = (int)std::min<long long>(32, std::max<long long>(1, (want + ctas - 1) / ctas));
        long long per = (c->N + split - 1) / split;
        if (per < best.tile) split = (int)std::max<long long>(1, c->N / best.tile);
        best.split = split;
        return best;
    };
    FarTune t32 = pick(true), t64 = pick(false);
    // double-float kernel: one target per thread, FP32-ALU bound like the FP32 kernel
    FarTune tdf{128, 1, 1, 128};
    {
        double best = 1e30;
        for (int th = 64; th <= 256; th += 64) {
            int chunks = (c->npn + th - 1) / th;
            double waste = (double)(chunks * th - c->npn) / c->npn + (th == 128 ? 0.0 : 0.001);
            if (waste < best - 1e-12) { best = waste; tdf.threads = th; }
        }
        int chunks = (c->npn + tdf.threads - 1) / tdf.threads;
        long long ctas = (long long)c->n * chunks;
        long long want = (long long)c->sm_count * 8;
        tdf.split = (int)std::min<long long>(16, std::max<long long>(1, (want + ctas - 1) / ctas));
        if ((c->N + tdf.split - 1) / tdf.split < tdf.tile) tdf.split = (int)std::max<long long>(1, c->N / tdf.tile);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int op = 0; op < 3; ++op) {
        c->tune32[op] = t32;
        c->tune64[op] = t64;
        c->tunedf[op] = tdf;
        auto it = g_tune_cache.find(std::make_tuple(c->n, c->p, c->sm_count, op, (int)kModeF32));
        if (it != g_tune_cache.end()) c->tune32[op] = it->second;
        it = g_tune_cache.find(std::make_tuple(c->n, c->p, c->sm_count, op, (int)kModeDF));
        if (it != g_tune_cache.end()) c->tunedf[op] = it->second;
    }
}

int max_split(const sbie_ctx* c) {
    int s = 1;
    for (int op = 0; op < 3; ++op)
        s = std::max(s, std::max(c->tune32[op].split, std::max(c->tune64[op].split, c->tunedf[op].split)));
    return s;
}

sbie_status ensure_part(sbie_ctx* c, int split_needed = 0) {
    size_t need = (size_t)std::max(max_split(c), split_needed) * c->N * 3;
    if (need <= c->part_cap) return SBIE_OK;
    if (c->d_part) cudaFree(c->d_part);
    c->d_part = nullptr;
    c->part_cap = 0;
    if (dmalloc(&c->d_part, need) != cudaSuccess) return fail(c, SBIE_ERR_OOM, "far-field partials");
    c->part_cap = need;
    return SBIE_OK;
}

// Arithmetic of the FP64-accurate operator of a context: native FP64 for
// SBIE_FP64, the double-float far field otherwise.
int hi_mode(const sbie_ctx* c) { return c->opts.prec == SBIE_FP64 ? kModeF64 : kModeDF; }

Kern kern_of(int op) {
    if (op == SBIE_OP_S) return Kern::S;
    if (op == SBIE_OP_D || op == SBIE_OP_RESISTANCE) return Kern::D;
    return Kern::K;
}

// out = A in, all device memory, on c->stream, in arithmetic `mode`
// (kModeF64, kModeF32 or kModeDF).
sbie_status apply_dev(sbie_ctx* c, int op, int mode, const double* in, double* out) {
    const Kern k = kern_of(op);
    const bool f32 = mode == kModeF32;
    {
        StageScope s(c, ST_FAR);
        CK(launch_pack(c, in, mode));
        CK(launch_far(c, k, mode, out));
        if (c->prof.on) (f32 ? c->prof.pairs_f32 : c->prof.pairs_f64) += far_pairs(c);
    }
    {
        StageScope s(c, ST_SELF);
        CK(launch_self(c, k, in, out, true, c->n_near > 0));
    }
    if (c->n_near > 0) {
        StageScope s(c, ST_NEAR);
        CK(launch_near(c, k, f32, out));
    }
    if (op == SBIE_OP_RESISTANCE || op == SBIE_OP_MOBILITY) {
        StageScope s(c, ST_COMPL);
        CK(launch_moments(c, in));
        if (op == SBIE_OP_RESISTANCE) CK(launch_completion(c, f32, out));
        CK(launch_finalize(c, op, in, out));
    }
    return SBIE_OK;
}

double nrm2(sbie_ctx* c, const double* v, long long n, sbie_status* st) {
    double r = 0.0;
    cudaError_t e = blas_dots(c, v, 1, n, v, n, &r);
    if (e != cudaSuccess) {
        c->err = std::string("norm: ") + cudaGetErrorString(e);
        *st = SBIE_ERR_CUDA;
        return 0.0;
    }
    *st = SBIE_OK;
    return std::sqrt(r);
}

sbie_status ensure_krylov(sbie_ctx* c, int m) {
    if (c->d_V && c->krylov_m >= m) return SBIE_OK;
    if (c->d_V) cudaFree(c->d_V);
    c->d_V = nullptr;
    if (dmalloc(&c->d_V, (size_t)(m + 1) * c->N * 3) != cudaSuccess) return fail(c, SBIE_ERR_OOM, "Krylov basis");
    c->krylov_m = m;
    return SBIE_OK;
}

struct GmresOut {
    int iters = 0, restarts = 0;
    double rel = 0.0;  // residual of the final iterate, recomputed with A
    bool converged = false;
};

// Restarted GMRES with classical Gram-Schmidt applied twice, x0 = 0.
// A(in, out) applies the operator to device vectors.  The residual at every
// restart (and at the end) is recomputed as b - A x.
sbie_status gmres(sbie_ctx* c, const std::function<sbie_status(const double*, double*)>& A, const double* b,
                  double* x, double tol, int restart, int max_iter, GmresOut& go) {
    const long long n3 = c->N * 3;
    restart = std::max(1, std::min(restart, 250));
    CKS(ensure_krylov(c, restart));
    sbie_status st;
    const double nb = nrm2(c, b, n3, &st);
    CKS(st);
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n3, c->stream));
    go = GmresOut();
    if (!(nb > 0.0)) {
        if (!std::isfinite(nb)) return fail(c, SBIE_ERR_NUMERIC, "right-hand side is not finite");
        go.converged = true;
        return SBIE_OK;
    }
    double* r = c->d_res;
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
    double beta = nb;
    std::vector<double> H((restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), h(restart + 1),
        h2(restart + 1), y(restart);
    double* d_h = c->d_red + 2 * 296 * 256;  // scratch for small device vectors (after dot partials)
    int total = 0;
    while (true) {
        if (beta / nb <= tol) {
            go.converged = true;
            break;
        }
        if (total >= max_iter) break;
        const int m = std::min(restart, max_iter - total);
        double* V = c->d_V;
        CK(blas_scale_copy(c, 1.0 / beta, r, V, n3));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int kd = 0;
        bool breakdown = false;
        for (int k = 0; k < m; ++k) {
            double* w = V + (size_t)(k + 1) * n3;
            CKS(A(V + (size_t)k * n3, w));
            {
                StageScope s(c, ST_BLAS);
                CK(blas_dots(c, V, k + 1, n3, w, n3, h.data()));
                std::memcpy(c->h_red + 256, h.data(), sizeof(double) * (k + 1));
                CK(cudaMemcpyAsync(d_h, c->h_red + 256, sizeof(double) * (k + 1), cudaMemcpyHostToDevice, c->stream));
                CK(blas_gemv_sub(c, V, k + 1, n3, d_h, w, n3));
                CK(blas_dots(c, V, k + 1, n3, w, n3, h2.data()));
                std::memcpy(c->h_red + 256, h2.data(), sizeof(double) * (k + 1));
                CK(cudaMemcpyAsync(d_h, c->h_red + 256, sizeof(double) * (k + 1), cudaMemcpyHostToDevice, c->stream));
                CK(blas_gemv_sub(c, V, k + 1, n3, d_h, w, n3));
            }
            for (int j = 0; j <= k; ++j) h[j] += h2[j];
            double hk1 = nrm2(c, w, n3, &st);
            CKS(st);
            if (!std::isfinite(hk1)) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf in the Krylov basis");
            if (hk1 > 0.0) CK(blas_scale_copy(c, 1.0 / hk1, w, w, n3));
            for (int j = 0; j < k; ++j) {
                double a0 = h[j], a1 = h[j + 1];
                h[j] = cs[j] * a0 + sn[j] * a1;
                h[j + 1] = -sn[j] * a0 + cs[j] * a1;
            }
            double den = std::hypot(h[k], hk1);
            cs[k] = den > 0 ? h[k] / den : 1.0;
            sn[k] = den > 0 ? hk1 / den : 0.0;
            h[k] = den;
            for (int j = 0; j <= k; ++j) H[j * restart + k] = h[j];
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            ++total;
            kd = k + 1;
            if (std::fabs(g[k + 1]) / nb <= tol) break;
            if (hk1 == 0.0) {
                breakdown = true;
                break;
            }
        }
        // back substitution for y, then x += V y
        for (int i = kd - 1; i >= 0; --i) {
            double s = g[i];
            for (int j = i + 1; j < kd; ++j) s -= H[i * restart + j] * y[j];
            y[i] = s / H[i * restart + i];
        }
        std::memcpy(c->h_red + 256, y.data(), sizeof(double) * kd);
        CK(cudaMemcpyAsync(d_h, c->h_red + 256, sizeof(double) * kd, cudaMemcpyHostToDevice, c->stream));
        CK(blas_gemv_add(c, V, kd, n3, d_h, x, n3));
        CKS(A(x, r));
        CK(blas_lincomb(c, 1.0, b, -1.0, r, r, n3));
        beta = nrm2(c, r, n3, &st);
        CKS(st);
        if (!std::isfinite(beta)) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf residual");
        ++go.restarts;
        if (breakdown && beta / nb > tol) break;
    }
    go.iters = total;
    go.rel = beta / nb;
    go.converged = go.rel <= tol;
    return SBIE_OK;
}

// Solve A x = b to the FP64 residual tolerance.  SBIE_FP64: GMRES on the FP64
// operator.  SBIE_MIXED: iterative refinement -- the residual b - A x with the
// FP64 operator, corrections by GMRES on the mixed-precision operator.
sbie_status solve_op(sbie_ctx* c, int op, const double* b, double* x, sbie_solve_info* info) {
    const long long n3 = c->N * 3;
    // FP64-accurate operator: native FP64, or the far field in double-float
    auto A64 = [&](const double* in, double* out) { return apply_dev(c, op, hi_mode(c), in, out); };
    auto A32 = [&](const double* in, double* out) { return apply_dev(c, op, kModeF32, in, out); };
    const double tol = c->opts.tol;
    GmresOut go;
    sbie_solve_info inf{};
    if (c->opts.prec != SBIE_MIXED) {
        CKS(gmres(c, A64, b, x, tol, c->opts.restart, c->opts.max_iter, go));
        inf.iters = go.iters;
        inf.restarts = go.restarts;
        inf.rel_residual_true = go.rel;
    } else {
        sbie_status st;
        const double nb = nrm2(c, b, n3, &st);
        CKS(st);
        CK(cudaMemsetAsync(x, 0, sizeof(double) * n3, c->stream));
        double* r = c->d_rhs == b ? c->d_tmp2 : c->d_rhs;
        CK(cudaMemcpyAsync(r, b, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
        double rel = nb > 0 ? 1.0 : 0.0;
        int iters = 0, outers = 0;
        double* d = c->d_xsol == x ? c->d_tmp : c->d_xsol;
        while (rel > tol && iters < c->opts.max_iter && outers < 20) {
            const double inner_tol = std::min(1e-3, std::max(1e-5, 0.5 * tol / rel));
            CKS(gmres(c, A32, r, d, inner_tol, c->opts.restart, c->opts.max_iter - iters, go));
            iters += go.iters;
            CK(blas_axpy(c, 1.0, d, x, n3));
            CKS(A64(x, r));
            CK(blas_lincomb(c, 1.0, b, -1.0, r, r, n3));
            double rn = nrm2(c, r, n3, &st);
            CKS(st);
            if (!std::isfinite(rn)) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf residual");
            ++outers;
            rel = rn / nb;
            if (go.iters == 0) break;
        }
        inf.iters = iters;
        inf.refinements = outers;
        inf.rel_residual_true = rel;
    }
    inf.n_near_pairs = c->n_near;
    if (info) {
        info->iters = inf.iters;
        info->restarts = inf.restarts;
        info->refinements = inf.refinements;
        info->rel_residual_true = inf.rel_residual_true;
        info->n_near_pairs = inf.n_near_pairs;
    }
    return inf.rel_residual_true <= tol ? SBIE_OK : SBIE_ERR_NOT_CONVERGED;
}

bool finite_all(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

extern "C" {

sbie_status sphere_bie_default_opts(sbie_opts* o) {
    if (!o) return SBIE_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->p = 8;
    o->eta = 1.0;
    o->prec = SBIE_FP64;
    o->tol = 1e-8;
    o->restart = 60;
    o->max_iter = 600;
    o->mem_kind = 0;
    o->stream = nullptr;
    return SBIE_OK;
}

sbie_status sphere_bie_create(int n, const double* centres, const double* radii, const sbie_opts* opts,
                              sbie_ctx** out) {
    if (!out) return fail(nullptr, SBIE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !centres || !radii || !opts) return fail(nullptr, SBIE_ERR_ARG, "need n >= 1 and non-NULL arrays");
    if (opts->p < 1 || opts->p > kMaxP) return fail(nullptr, SBIE_ERR_ARG, "p must be in [1, 24]");
    if (!(opts->eta >= 0.0) || !std::isfinite(opts->eta)) return fail(nullptr, SBIE_ERR_ARG, "eta must be >= 0");
    if (opts->prec != SBIE_FP64 && opts->prec != SBIE_MIXED && opts->prec != SBIE_FP64_DF)
        return fail(nullptr, SBIE_ERR_ARG, "bad precision");
    if (opts->mem_kind != 0 && opts->mem_kind != 1) return fail(nullptr, SBIE_ERR_ARG, "mem_kind must be 0 or 1");
    if (opts->use_learned_precond != 0) return fail(nullptr, SBIE_ERR_ARG, "learned preconditioner not available");
    if (!(opts->tol > 0.0) || opts->restart < 1 || opts->max_iter < 0)
        return fail(nullptr, SBIE_ERR_ARG, "need tol > 0, restart >= 1, max_iter >= 0");
    if (!finite_all(centres, (size_t)n * 3) || !finite_all(radii, n))
        return fail(nullptr, SBIE_ERR_ARG, "non-finite centre or radius");
    for (int i = 0; i < n; ++i)
        if (!(radii[i] > 0.0)) return fail(nullptr, SBIE_ERR_ARG, "radii must be positive");

    sbie_ctx* c = new (std::nothrow) sbie_ctx();
    if (!c) return fail(nullptr, SBIE_ERR_OOM, "host allocation");
    c->opts = *opts;
    c->n = n;
    c->p = opts->p;
    c->nlat = c->p + 1;
    c->nlon = 2 * c->p + 2;
    c->npn = c->nlat * c->nlon;
    c->N = (long long)n * c->npn;
    c->h_c.assign(centres, centres + 3 * (size_t)n);
    c->h_a.assign(radii, radii + n);

    // close pairs (negation of Eq. 4.5) and overlap check
    c->h_near_ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < n; ++k) {
            if (k == i) continue;
            double dx = centres[3 * i] - centres[3 * k], dy = centres[3 * i + 1] - centres[3 * k + 1],
                   dz = centres[3 * i + 2] - centres[3 * k + 2];
            double gap = std::sqrt(dx * dx + dy * dy + dz * dz) - radii[i] - radii[k];
            if (gap <= 0.0) {
                g_last_error = "spheres " + std::to_string(i) + " and " + std::to_string(k) + " overlap or touch";
                delete c;
                return SBIE_ERR_OVERLAP;
            }
            if (gap < opts->eta * 2.0 * std::max(radii[i], radii[k])) c->h_near_idx.push_back(k);
        }
        c->h_near_ptr[i + 1] = (int)c->h_near_idx.size();
    }
    c->n_near = (long long)c->h_near_idx.size();

    auto bail = [&](sbie_status s, const std::string& m) {
        g_last_error = m;
        free_all(c);
        delete c;
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
    c->sm_count = prop.multiProcessorCount;
    if (opts->stream) {
        c->stream = (cudaStream_t)opts->stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        c->own_stream = true;
    }
    c->tl = tab_layout(c->p);
    std::vector<double> htab;
    build_tables(c->p, htab);
    const long long N = c->N;
    const int P1 = c->p + 1;
    const int Kc = sh_count(c->p + 2);
    bool ok = true;
    ok &= dmalloc(&c->d_c, 3 * (size_t)n) == cudaSuccess;
    ok &= dmalloc(&c->d_a, (size_t)n) == cudaSuccess;
    ok &= dmalloc(&c->d_x, 4 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_xhi, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_xlo, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_nrm, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_nrm64, 4 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_sph, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_near_ptr, (size_t)n + 1) == cudaSuccess;
    ok &= dmalloc(&c->d_near_idx, (size_t)std::max<long long>(1, c->n_near)) == cudaSuccess;
    ok &= dmalloc(&c->d_tab, (size_t)c->tl.total) == cudaSuccess;
    ok &= dmalloc(&c->d_coef, (size_t)n * 3 * P1 * P1 * 2) == cudaSuccess;
    if (c->n_near > 0) {
        ok &= dmalloc(&c->d_chan, (size_t)n * Kc * kTracChannels) == cudaSuccess;
        ok &= dmalloc(&c->d_chanf, (size_t)n * Kc * 28) == cudaSuccess;
    }
    ok &= dmalloc(&c->d_mom, 6 * (size_t)n) == cudaSuccess;
    ok &= dmalloc(&c->d_src64, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_srcf, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_in, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_out, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_tmp, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_tmp2, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_xsol, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_rhs, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_res, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_small, 3 * (size_t)n * 6 + 32) == cudaSuccess;
    ok &= dmalloc(&c->d_red, (size_t)4 * 296 * 256) == cudaSuccess;
    ok &= cudaMallocHost(reinterpret_cast<void**>(&c->h_red), sizeof(double) * 1024) == cudaSuccess;
    if (!ok) return bail(SBIE_ERR_OOM, "device allocation failed");
    choose_tuning(c);
    {
        sbie_status s = ensure_part(c);
        if (s != SBIE_OK) return bail(s, c->err);
    }
    e = cudaMemcpy(c->d_c, centres, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_a, radii, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_near_ptr, c->h_near_ptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->n_near > 0)
        e = cudaMemcpy(c->d_near_idx, c->h_near_idx.data(), sizeof(int) * c->n_near, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_tab, htab.data(), sizeof(double) * htab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_geometry(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    c->err = "no error";
    *out = c;
    return SBIE_OK;
}

sbie_status sphere_bie_num_nodes(const sbie_ctx* c, long long* n_nodes) {
    if (!c || !n_nodes) return SBIE_ERR_ARG;
    *n_nodes = c->N;
    return SBIE_OK;
}

sbie_status sphere_bie_nodes(const sbie_ctx* cc, double* xyz, double* normals, double* weights) {
    sbie_ctx* c = const_cast<sbie_ctx*>(cc);
    if (!c) return SBIE_ERR_ARG;
    std::vector<double> x4(4 * (size_t)c->N), n4(4 * (size_t)c->N);
    CK(cudaMemcpy(x4.data(), c->d_x, sizeof(double) * x4.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(n4.data(), c->d_nrm64, sizeof(double) * n4.size(), cudaMemcpyDeviceToHost));
    for (long long i = 0; i < c->N; ++i) {
        for (int d = 0; d < 3; ++d) {
            if (xyz) xyz[3 * i + d] = x4[4 * i + d];
            if (normals) normals[3 * i + d] = n4[4 * i + d];
        }
        if (weights) weights[i] = x4[4 * i + 3];
    }
    return SBIE_OK;
}

sbie_status sphere_bie_apply_operator(sbie_ctx* c, sbie_op op, const double* density, double* out) {
    if (!c) return SBIE_ERR_ARG;
    if (!density || !out) return fail(c, SBIE_ERR_ARG, "NULL density or out");
    if (op < SBIE_OP_S || op > SBIE_OP_RESISTANCE) return fail(c, SBIE_ERR_ARG, "bad operator");
    if (density == out) return fail(c, SBIE_ERR_ARG, "density and out must not alias");
    const int mode = c->opts.prec == SBIE_MIXED ? kModeF32 : hi_mode(c);
    const size_t bytes = sizeof(double) * 3 * (size_t)c->N;
    if (c->opts.mem_kind == 0) {
        CK(cudaMemcpyAsync(c->d_in, density, bytes, cudaMemcpyHostToDevice, c->stream));
        CKS(apply_dev(c, op, mode, c->d_in, c->d_out));
        CK(cudaMemcpyAsync(out, c->d_out, bytes, cudaMemcpyDeviceToHost, c->stream));
    } else {
        CKS(apply_dev(c, op, mode, density, out));
    }
    CK(cudaStreamSynchronize(c->stream));
    return SBIE_OK;
}

sbie_status sphere_bie_solve_mobility(sbie_ctx* c, const double* forces, const double* torques, double* vel,
                                      double* omega, sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!forces || !torques || !vel || !omega) return fail(c, SBIE_ERR_ARG, "NULL argument");
    auto t0 = std::chrono::steady_clock::now();
    const size_t sb = sizeof(double) * 3 * c->n;
    const long long n3 = c->N * 3;
    double* dF = c->d_small;
    double* dT = dF + 3 * c->n;
    double* dv = dT + 3 * c->n;
    double* dw = dv + 3 * c->n;
    const double *F = forces, *T = torques;
    if (c->opts.mem_kind == 0) {
        CK(cudaMemcpyAsync(dF, forces, sb, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dT, torques, sb, cudaMemcpyHostToDevice, c->stream));
        F = dF;
        T = dT;
    }
    double* rho = c->d_tmp;
    double* b = c->d_rhs;
    double* mu = c->d_xsol;
    CK(launch_rho(c, F, T, rho));
    // b = -(1/2 I + K) rho
    CKS(apply_dev(c, SBIE_OP_K, hi_mode(c), rho, b));
    CK(blas_lincomb(c, -0.5, rho, -1.0, b, b, n3));
    // keep rho: solve_op uses d_tmp in mixed mode, so copy it aside
    double* rho_keep = c->d_in;
    CK(cudaMemcpyAsync(rho_keep, rho, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
    sbie_solve_info inf{};
    sbie_status st = solve_op(c, SBIE_OP_MOBILITY, b, mu, &inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    // u = S[mu + rho] on every sphere; rigid projection
    CK(blas_lincomb(c, 1.0, mu, 1.0, rho_keep, c->d_tmp2, n3));
    CKS(apply_dev(c, SBIE_OP_S, hi_mode(c), c->d_tmp2, c->d_out));
    double* V = c->opts.mem_kind == 0 ? dv : vel;
    double* W = c->opts.mem_kind == 0 ? dw : omega;
    CK(launch_rigid_projection(c, c->d_out, V, W));
    if (c->opts.mem_kind == 0) {
        CK(cudaMemcpyAsync(vel, dv, sb, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(omega, dw, sb, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return st;
}

sbie_status sphere_bie_solve_resistance(sbie_ctx* c, const double* vel, const double* omega, const double* bg_u0,
                                        const double* bg_grad, double* forces, double* torques, sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!vel || !omega || !forces || !torques) return fail(c, SBIE_ERR_ARG, "NULL argument");
    auto t0 = std::chrono::steady_clock::now();
    const size_t sb = sizeof(double) * 3 * c->n;
    double* dv = c->d_small;
    double* dw = dv + 3 * c->n;
    const double *V = vel, *W = omega;
    if (c->opts.mem_kind == 0) {
        CK(cudaMemcpyAsync(dv, vel, sb, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dw, omega, sb, cudaMemcpyHostToDevice, c->stream));
        V = dv;
        W = dw;
    }
    if (bg_u0 && !finite_all(bg_u0, 3)) return fail(c, SBIE_ERR_ARG, "non-finite u0");
    if (bg_grad && !finite_all(bg_grad, 9)) return fail(c, SBIE_ERR_ARG, "non-finite velocity gradient");
    double* b = c->d_rhs;
    double* psi = c->d_xsol;
    CK(launch_resistance_rhs(c, V, W, bg_u0, bg_grad, b));
    sbie_solve_info inf{};
    sbie_status st = solve_op(c, SBIE_OP_RESISTANCE, b, psi, &inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    CK(launch_moments(c, psi));
    // forces / torques from the moments [n][6]
    double* dF = c->d_small + 6 * c->n;
    double* dT = dF + 3 * c->n;
    CK(cudaMemcpy2DAsync(c->opts.mem_kind == 0 ? dF : forces, sizeof(double) * 3, c->d_mom, sizeof(double) * 6,
                         sizeof(double) * 3, c->n, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpy2DAsync(c->opts.mem_kind == 0 ? dT : torques, sizeof(double) * 3, c->d_mom + 3, sizeof(double) * 6,
                         sizeof(double) * 3, c->n, cudaMemcpyDeviceToDevice, c->stream));
    if (c->opts.mem_kind == 0) {
        CK(cudaMemcpyAsync(forces, dF, sb, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(torques, dT, sb, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return st;
}

sbie_status sphere_bie_destroy(sbie_ctx* c) {
    if (!c) return SBIE_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
    return SBIE_OK;
}

const char* sphere_bie_last_error(const sbie_ctx* c) {
    return c ? c->err.c_str() : g_last_error.c_str();
}

}  // extern "C"

namespace {

// Times every admissible tiling of one far-field kernel; keeps the fastest.
sbie_status tune_one(sbie_ctx* c, Kern k, int mode, sbie_far_tuning* chosen) {
    struct Cand { FarTune t; float ms; };
    std::vector<Cand> cands;
    const bool f32 = mode == kModeF32;
    const int tpts32[2] = {2, 4}, tpts1[1] = {1};
    const int* tpts = f32 ? tpts32 : tpts1;
    const int ntpt = f32 ? 2 : 1;
    const int ths32[5] = {64, 96, 128, 192, 256}, thsdf[3] = {64, 128, 256};
    const int* ths = f32 ? ths32 : thsdf;
    const int nth = f32 ? 5 : 3;
    const int splits32[8] = {1, 2, 3, 4, 6, 8, 12, 16}, splitsdf[4] = {1, 2, 4, 8};
    const int* splits = f32 ? splits32 : splitsdf;
    const int nsp = f32 ? 8 : 4;
    const int tiles32[2] = {128, 256}, tilesdf[1] = {128};
    const int* tiles = f32 ? tiles32 : tilesdf;
    const int nti = f32 ? 2 : 1;
    for (int a = 0; a < ntpt; ++a)
        for (int b = 0; b < nth; ++b) {
            const int tpt = tpts[a], th = ths[b];
            int slots = th * tpt;
            int chunks = (c->npn + slots - 1) / slots;
            double waste = (double)(chunks * slots - c->npn) / c->npn;
            if (waste > 0.30) continue;
            for (int s = 0; s < nsp; ++s) {
                const int sp = splits[s];
                long long ctas = (long long)c->n * chunks * sp;
                if (ctas < c->sm_count && s != 0) continue;
                if (ctas > 64LL * c->sm_count) continue;
                for (int t = 0; t < nti; ++t) {
                    if ((c->N + sp - 1) / sp < tiles[t]) continue;
                    cands.push_back(Cand{FarTune{th, tpt, sp, tiles[t]}, 0.f});
                }
            }
        }
    FarTune* slot = f32 ? &c->tune32[(int)k] : &c->tunedf[(int)k];
    if (cands.empty()) cands.push_back(Cand{*slot, 0.f});
    float dummy;
    CK(time_far(c, k, mode, cands[0].t, &dummy));  // warm-up
    for (auto& cd : cands) CK(time_far(c, k, mode, cd.t, &cd.ms));
    std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    const size_t top = std::min<size_t>(f32 ? 6 : 3, cands.size());
    for (size_t i = 0; i < top; ++i) {
        float best = cands[i].ms;
        for (int r = 0; r < 2; ++r) {
            float ms;
            CK(time_far(c, k, mode, cands[i].t, &ms));
            best = std::min(best, ms);
        }
        cands[i].ms = best;
    }
    std::sort(cands.begin(), cands.begin() + top, [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    *slot = cands[0].t;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[std::make_tuple(c->n, c->p, c->sm_count, (int)k, mode)] = cands[0].t;
    }
    if (chosen) {
        chosen->threads = cands[0].t.threads;
        chosen->targets_per_thread = cands[0].t.tpt;
        chosen->split = cands[0].t.split;
        chosen->tile = cands[0].t.tile;
        chosen->ms = cands[0].ms;
        chosen->candidates = (int)cands.size();
    }
    return SBIE_OK;
}

}  // namespace

extern "C" {

sbie_status sphere_bie_autotune(sbie_ctx* c, sbie_op op, sbie_far_tuning* chosen) {
    if (!c) return SBIE_ERR_ARG;
    if (op < SBIE_OP_S || op > SBIE_OP_RESISTANCE) return fail(c, SBIE_ERR_ARG, "bad operator");
    const Kern k = kern_of(op);
    CKS(ensure_part(c, 16));
    CK(cudaMemsetAsync(c->d_srcf, 0, sizeof(float4) * c->N, c->stream));
    CK(cudaMemsetAsync(c->d_src64, 0, sizeof(double4) * c->N, c->stream));
    if (chosen) std::memset(chosen, 0, 2 * sizeof(*chosen));
    if (c->opts.prec == SBIE_MIXED) CKS(tune_one(c, k, kModeF32, chosen));
    if (c->opts.prec != SBIE_FP64) CKS(tune_one(c, k, kModeDF, chosen ? chosen + 1 : nullptr));
    return SBIE_OK;
}

sbie_status sphere_bie_profile(sbie_ctx* c, int enable) {
    if (!c) return SBIE_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    c->prof.on = enable != 0;
    for (int s = 0; s < 8; ++s) {
        c->prof.ms[s] = 0;
        c->prof.launches[s] = 0;
        c->prof_used[s] = 0;
    }
    c->prof.pairs_f32 = c->prof.pairs_f64 = 0;
    c->prof.kernels0 = c->n_launch;
    return SBIE_OK;
}

sbie_status sphere_bie_profile_read(sbie_ctx* c, sbie_profile* out) {
    if (!c || !out) return SBIE_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < 8; ++s) {
        for (int i = 0; i < c->prof_used[s]; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->prof_events[s][i].first, c->prof_events[s][i].second));
            c->prof.ms[s] += ms;
            c->prof.launches[s] += 1;
        }
        c->prof_used[s] = 0;
    }
    std::memset(out, 0, sizeof(*out));
    for (int s = 0; s < 8; ++s) {
        out->ms[s] = c->prof.ms[s];
        out->launches[s] = c->prof.launches[s];
    }
    out->far_pairs_f32 = c->prof.pairs_f32;
    out->far_pairs_f64 = c->prof.pairs_f64;
    out->kernel_launches = c->n_launch - c->prof.kernels0;
    return SBIE_OK;
}

}  // extern "C"
