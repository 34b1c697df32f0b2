// C interface (include/sphere_bie.h): context lifetime, operator assembly
// (Sec. 4.3), GMRES on the device and the mobility (Eq. 5.8) and resistance
// (Eq. 5.19) drivers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <atomic>
#include <map>
#include <thread>
#include <utility>
#include <mutex>
#include <new>
#include <tuple>
#include <fstream>
#include <random>

#include "common.h"
#include "mlp.h"

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

// Host <-> device copies ordered on a (non-blocking) stream.  A plain
// cudaMemcpy runs on the legacy default stream, which is not ordered with
// non-blocking streams, so every copy of a context goes through these.
template <typename T>
cudaError_t h2d(cudaStream_t s, T* dst, const T* src, size_t count) {
    return cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s);
}

template <typename T>
cudaError_t d2h(cudaStream_t s, T* dst, const T* src, size_t count) {
    cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

// Captured restart cycles bake in device addresses and far-field tilings;
// every reallocation or retuning advances this counter and a cycle graph
// recorded under an older value is captured again before its next use.
std::atomic<unsigned long long> g_graph_epoch{1};

void drop_graphs(sbie_ctx* c) {
    for (CycleGraph& g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    c->graphs.clear();
}

void free_all(sbie_ctx* c) {
    drop_graphs(c);
    self_gemm_free(c);
    for (sbie_ctx* q : c->parts) {
        free_all(q);
        delete q;
    }
    c->parts.clear();
    void* ptrs[] = {c->d_c, c->d_a, c->d_x, c->d_xhi, c->d_xlo, c->d_nrm, c->d_nrm64, c->d_sph, c->d_near_ptr,
                    c->d_near_idx, c->d_tab, c->d_coef, c->d_chan, c->d_chanf, c->d_mom, c->d_part, c->d_src64,
                    c->d_srcf, c->d_in, c->d_out, c->d_tmp, c->d_tmp2, c->d_small, c->d_red, c->d_V, c->d_xsol,
                    c->d_rhs, c->d_res, c->d_prob_sph, c->d_sph_prob, c->d_node_prob, c->d_seg3, c->d_H, c->d_pvec,
                    c->d_ZS, c->d_ZSf, c->d_ZA, c->d_modes, c->d_low, c->d_lowe, c->d_pz, c->d_ad, c->d_adi, c->d_vk,
                    c->d_sq, c->d_lcoef, c->d_rotp, c->d_rotm, c->d_fgeo, c->d_fcoef, c->d_fchan, c->d_fblk,
                    c->d_fiota, c->d_tabf, c->d_rotpf, c->d_rotmf, c->d_fcoeff, c->d_fchanf, c->d_fblkf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (PrecState& P : c->prec)
        for (void* p : {(void*)P.d_pp_ptr, (void*)P.d_pp_idx, (void*)P.d_pp_pair, (void*)P.d_pinv, (void*)P.d_sinv,
                        (void*)P.d_pp_own, (void*)P.d_cpart})
            if (p) cudaFree(p);
    if (c->h_red) cudaFreeHost(c->h_red);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->h_pack) cudaFreeHost(c->h_pack);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (auto& v : c->prof_events)
        for (auto& pr : v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Buffers and per-entry frames of the rotated close-pair scheme (Sec. 4.2): for
// entry e (target i, source k = near_idx[e]) the frame's pole points from c_k to
// c_i, (sin b cos a, sin b sin a, cos b); a = 0 on the polar axis.
sbie_status setup_near_fft(sbie_ctx* c, const std::vector<double>& htab) {
    const long long ne = c->n_near;
    const int P1 = c->p + 1, S = P1 * P1;
    std::vector<double> Mp, Mm;
    rotx90_tables(c->p, Mp, Mm);
    std::vector<double> geo((size_t)ne * 8, 0.0);
    std::vector<int> iota((size_t)ne + 1);
    for (long long q = 0; q <= ne; ++q) iota[q] = (int)q;
    for (int i = 0; i < c->n; ++i)
        for (int e = c->h_near_ptr[i]; e < c->h_near_ptr[i + 1]; ++e) {
            const int k = c->h_near_idx[e];
            const double vx = c->h_c[3 * i] - c->h_c[3 * k], vy = c->h_c[3 * i + 1] - c->h_c[3 * k + 1],
                         vz = c->h_c[3 * i + 2] - c->h_c[3 * k + 2];
            const double d = std::sqrt(vx * vx + vy * vy + vz * vz), rxy = std::sqrt(vx * vx + vy * vy);
            double* g = geo.data() + 8 * (size_t)e;
            g[0] = rxy > 0 ? vx / rxy : 1.0;   // cos a
            g[1] = rxy > 0 ? vy / rxy : 0.0;   // sin a
            g[2] = vz / d;                     // cos b
            g[3] = rxy / d;                    // sin b
            g[4] = d / c->h_a[k];
            g[5] = c->h_a[i] / c->h_a[k];
            g[6] = c->h_a[k];
        }
    const size_t Kt = (size_t)sh_count(c->p + 2);
    bool ok = dmalloc(&c->d_rotp, Mp.size()) == cudaSuccess && dmalloc(&c->d_rotm, Mm.size()) == cudaSuccess &&
              dmalloc(&c->d_fgeo, geo.size()) == cudaSuccess &&
              dmalloc(&c->d_fcoef, (size_t)ne * 6 * S) == cudaSuccess &&
              dmalloc(&c->d_fchan, (size_t)ne * Kt * kTracChannels) == cudaSuccess &&
              dmalloc(&c->d_fblk, (size_t)ne * 6 * S) == cudaSuccess && dmalloc(&c->d_fiota, iota.size()) == cudaSuccess;
    // FP32 copies for the FP32 operator of the mixed path
    std::vector<float> tabf, Mpf, Mmf;
    if (ok && c->opts.prec == SBIE_MIXED) {
        tabf.assign(htab.begin(), htab.end());
        Mpf.assign(Mp.begin(), Mp.end());
        Mmf.assign(Mm.begin(), Mm.end());
        ok = dmalloc(&c->d_tabf, tabf.size()) == cudaSuccess && dmalloc(&c->d_rotpf, Mpf.size()) == cudaSuccess &&
             dmalloc(&c->d_rotmf, Mmf.size()) == cudaSuccess &&
             dmalloc(&c->d_fcoeff, (size_t)ne * 6 * S) == cudaSuccess &&
             dmalloc(&c->d_fchanf, (size_t)ne * Kt * ((kTracChannels + 3) / 4 * 4)) == cudaSuccess &&
             dmalloc(&c->d_fblkf, (size_t)ne * 6 * S) == cudaSuccess;
    }
    if (!ok) return fail(c, SBIE_ERR_OOM, "rotated close-pair buffers");
    cudaError_t e = h2d(c->stream, c->d_rotp, Mp.data(), Mp.size());
    if (e == cudaSuccess && !tabf.empty()) e = h2d(c->stream, c->d_tabf, tabf.data(), tabf.size());
    if (e == cudaSuccess && !Mpf.empty()) e = h2d(c->stream, c->d_rotpf, Mpf.data(), Mpf.size());
    if (e == cudaSuccess && !Mmf.empty()) e = h2d(c->stream, c->d_rotmf, Mmf.data(), Mmf.size());
    if (e == cudaSuccess) e = h2d(c->stream, c->d_rotm, Mm.data(), Mm.size());
    if (e == cudaSuccess) e = h2d(c->stream, c->d_fgeo, geo.data(), geo.size());
    if (e == cudaSuccess) e = h2d(c->stream, c->d_fiota, iota.data(), iota.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SBIE_ERR_CUDA, std::string("rotated close pairs: ") + cudaGetErrorString(e));
    return SBIE_OK;
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
                // FP32: 64 threads x 4 targets (the 128-register build, 8
                // resident CTAs per SM) is what the autotuner settles on
                double pref = f32 ? ((tpt == 4 && th == 64) ? 0.0 : (tpt == 2 ? 0.03 : 0.04))
                                  : (tpt == 1 ? 0.0 : 0.05);
                pref += (th == 128 || (f32 && th == 64)) ? 0.0 : 0.001;
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
        if (f32 && best.threads == 64 && best.tpt == 4) {
            // about three whole waves of resident CTAs
            best.minb = 8;
            const int occ = far_occupancy(c, Kern::D, kModeF32, best);
            if (occ > 0) split = (int)std::min<long long>(32, std::max<long long>(1, 3LL * occ * c->sm_count / ctas));
        }
        // small contexts: shorter tiles before fewer splits
        while (best.tile > 32 && (c->N + split - 1) / split < best.tile) best.tile /= 2;
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
        while (tdf.tile > 32 && (c->N + tdf.split - 1) / tdf.split < tdf.tile) tdf.tile /= 2;
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
    ++g_graph_epoch;
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

sbie_status apply_dev(sbie_ctx* c, int op, int mode, const double* in, double* out);

// Operator of the magnetostatic equation (Eq. 5.13) on scalar densities held
// in component 0; internal (reached through sphere_bie_solve_mhd).
constexpr int kOpMagnetic = 7;

// Porous-media operator 1/2 I + S + D (Eq. 5.4): both layers' far fields,
// self terms and close-pair corrections, added.
sbie_status apply_porous(sbie_ctx* c, int mode, const double* in, double* out) {
    const bool f32 = mode == kModeF32;
    const bool far = c->far_pair_count > 0;
    const bool gemm = f32 && self_gemm_ready(c, kSelfS) && self_gemm_ready(c, kSelfDK);
    if (gemm) {
        StageScope s(c, ST_SELF);
        CK(launch_self_gemm(c, kSelfS, in, out, false));
        CK(launch_self_gemm(c, kSelfDK, in, out, true));
        if (c->n_near > 0) CK(launch_self_analysis(c, in));
    }
    if (far) {
        StageScope s(c, ST_FAR);
        CK(launch_pack(c, in, mode));
        CK(launch_far(c, Kern::S, mode, out, gemm));
        CK(launch_far(c, Kern::D, mode, out, true));
        if (c->prof.on) (f32 ? c->prof.pairs_f32 : c->prof.pairs_f64) += 2 * c->far_pair_count;
    }
    if (!gemm) {
        StageScope s(c, ST_SELF);
        CK(launch_self(c, Kern::S, in, out, far, c->n_near > 0));
        CK(launch_self(c, Kern::D, in, out, true, false));
    }
    if (c->n_near > 0) {
        StageScope s(c, ST_NEAR);
        if (c->opts.near_scheme == 1) {
            CK(launch_near_fft(c, Kern::S, f32, out));
            CK(launch_near_fft(c, Kern::D, f32, out));
        } else {
            CK(launch_near(c, Kern::S, f32, out));
            CK(launch_near(c, Kern::D, f32, out));
        }
    }
    StageScope s(c, ST_COMPL);
    CK(launch_finalize(c, SBIE_OP_POROUS, in, out));
    return SBIE_OK;
}

// out = A in, all device memory, on c->stream, in arithmetic `mode`
// (kModeF64, kModeF32 or kModeDF).
sbie_status apply_dev(sbie_ctx* c, int op, int mode, const double* in, double* out) {
    if (op == SBIE_OP_POROUS) return apply_porous(c, mode, in, out);
    if (op == kOpMagnetic) {
        // (1/2 I + eta K^L) on component 0 (the scalar density), 1/2 I on the
        // two unused components (FP64 in every precision mode)
        CK(laplace_apply(c, kLapKL, in, out));
        StageScope s(c, ST_COMPL);
        CK(launch_magnetic_finalize(c, c->mag_eta, in, out));
        return SBIE_OK;
    }
    if (op == SBIE_OP_SQUIRMER) {
        // (1/2 I + S + D)(in - P in) - P in, P the rigid projection per sphere
        if (!c->d_sq) return fail(c, SBIE_ERR_ARG, "squirmer buffers not allocated");
        double* q = c->d_sq;
        double* r = c->d_sq + 3 * c->N;
        {
            StageScope s(c, ST_COMPL);
            CK(launch_moments(c, in));
            CK(launch_rigid_split(c, in, q, r));
        }
        CKS(apply_porous(c, mode, q, out));
        StageScope s(c, ST_COMPL);
        CK(blas_axpy(c, -1.0, r, out, 3 * c->N));
        return SBIE_OK;
    }
    const Kern k = kern_of(op);
    const bool f32 = mode == kModeF32;
    // a context whose pairs are all close (the two-sphere probe problems of
    // the pair preconditioner) has no far field: the self term writes `out`
    const bool far = c->far_pair_count > 0;
    const int which = k == Kern::S ? kSelfS : kSelfDK;
    if (f32 && self_gemm_ready(c, which)) {
        // FP32 operator: the self term by the 3xTF32 GEMM writes `out` first
        // and the far field's reduction adds to it (the GEMM's epilogue then
        // needs no FP64 add); the close pairs keep FP64 VSH coefficients
        {
            StageScope s(c, ST_SELF);
            CK(launch_self_gemm(c, which, in, out, false));
            if (c->n_near > 0) CK(launch_self_analysis(c, in));
        }
        if (far) {
            StageScope s(c, ST_FAR);
            CK(launch_pack(c, in, mode));
            CK(launch_far(c, k, mode, out, true));
            c->prof.pairs_f32 += c->prof.on ? c->far_pair_count : 0;
        }
    } else {
        if (far) {
            StageScope s(c, ST_FAR);
            CK(launch_pack(c, in, mode));
            CK(launch_far(c, k, mode, out));
            if (c->prof.on) (f32 ? c->prof.pairs_f32 : c->prof.pairs_f64) += c->far_pair_count;
        }
        StageScope s(c, ST_SELF);
        CK(launch_self(c, k, in, out, far, c->n_near > 0));
    }
    if (c->n_near > 0) {
        StageScope s(c, ST_NEAR);
        CK(c->opts.near_scheme == 1 ? launch_near_fft(c, k, f32, out) : launch_near(c, k, f32, out));
    }
    if (op == SBIE_OP_RESISTANCE || op == SBIE_OP_MOBILITY) {
        StageScope s(c, ST_COMPL);
        CK(launch_moments(c, in));
        if (op == SBIE_OP_RESISTANCE) CK(launch_completion(c, f32, out));
        CK(launch_finalize(c, op, in, out));
    }
    return SBIE_OK;
}

// ---- system view: the parts (one per VSH order) and the problem segments of
// a context's vector.  A single-order context is its own only part.
struct Sys {
    sbie_ctx* top;
    std::vector<sbie_ctx*> parts;
    std::vector<long long> off3;
    long long n3;
    int P;
};

Sys sys_of(sbie_ctx* c) {
    Sys s;
    s.top = c;
    if (c->is_batch) {
        s.parts = c->parts;
        s.off3 = c->part_off3;
    } else {
        s.parts = {c};
        s.off3 = {0};
    }
    s.n3 = c->N * 3;
    s.P = (int)c->seg3.size() - 1;
    return s;
}

// The FP32 operator's self term is a tensor-core GEMM whose matrices (single
// layer; double layer = traction) are probed by the FP64 self kernel the first
// time a mixed-precision context applies or solves, before any graph capture.
sbie_status ensure_self_gemm(const Sys& S) {
    for (sbie_ctx* q : S.parts) {
        if (q->opts.prec != SBIE_MIXED) continue;
        cudaError_t e = self_gemm_build(q, kSelfS);
        if (e == cudaSuccess) e = self_gemm_build(q, kSelfDK);
        if (e != cudaSuccess)
            return fail(S.top, SBIE_ERR_CUDA, std::string("self-term matrices: ") + cudaGetErrorString(e));
    }
    return SBIE_OK;
}

// Work vectors of the squirmer operator, allocated before any graph capture.
sbie_status ensure_squirmer_buffers(const Sys& S) {
    for (sbie_ctx* q : S.parts)
        if (!q->d_sq && dmalloc(&q->d_sq, 6 * (size_t)q->N) != cudaSuccess)
            return fail(S.top, SBIE_ERR_OOM, "squirmer buffers");
    return SBIE_OK;
}

// Device flag of the self-term GEMMs (a bounded wait that ran out).
sbie_status check_self_gemm(const Sys& S) {
    for (sbie_ctx* q : S.parts) {
        int flag = 0;
        cudaError_t e = self_gemm_error(q, &flag);
        if (e != cudaSuccess) return fail(S.top, SBIE_ERR_CUDA, cudaGetErrorString(e));
        if (flag) return fail(S.top, SBIE_ERR_TIMEOUT, "self-term GEMM: a pipeline wait timed out");
    }
    return SBIE_OK;
}

sbie_status apply_sys(const Sys& S, int op, int mode, const double* in, double* out) {
    for (size_t i = 0; i < S.parts.size(); ++i) {
        sbie_status st = apply_dev(S.parts[i], op, mode, in + S.off3[i], out + S.off3[i]);
        if (st != SBIE_OK) {
            if (S.parts[i] != S.top) S.top->err = S.parts[i]->err;
            return st;
        }
    }
    return SBIE_OK;
}

sbie_status ensure_krylov(sbie_ctx* c, int m, int P) {
    const int B = seg_blocks(c->N * 3, P);
    const long long n3 = c->N * 3;
    if (!c->d_V || c->krylov_m < m) {
        if (c->d_V) cudaFree(c->d_V);
        c->d_V = nullptr;
        c->krylov_m = 0;
        if (dmalloc(&c->d_V, (size_t)(m + 1) * n3) != cudaSuccess) return fail(c, SBIE_ERR_OOM, "Krylov basis");
        c->krylov_m = m;
        ++g_graph_epoch;
    }
    if (!c->d_ad || c->ad.m < m || c->ad.P < P) {
        for (void* q : {(void*)c->d_ad, (void*)c->d_adi, (void*)c->d_vk})
            if (q) cudaFree(q);
        if (c->h_st) cudaFreeHost(c->h_st);
        if (c->h_pack) cudaFreeHost(c->h_pack);
        c->d_ad = nullptr;
        c->d_adi = nullptr;
        c->d_vk = nullptr;
        c->h_st = nullptr;
        c->h_pack = nullptr;
        c->ad = ArnoldiDev();
        const size_t Pm = (size_t)P * m, Pm1 = (size_t)P * (m + 1);
        const size_t nd = 4 * (size_t)P + Pm1 * m + 2 * Pm + Pm1 + 2 * Pm1 + Pm + (4 * (size_t)P + 1) + n3;
        if (dmalloc(&c->d_ad, nd) != cudaSuccess || dmalloc(&c->d_adi, kStWords + 2 * (size_t)P) != cudaSuccess ||
            dmalloc(&c->d_vk, (size_t)n3) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&c->h_st), sizeof(int) * kStWords) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&c->h_pack), sizeof(double) * (4 * (size_t)P + 1)) != cudaSuccess)
            return fail(c, SBIE_ERR_OOM, "GMRES cycle state");
        ArnoldiDev& A = c->ad;
        A.m = m;
        A.P = P;
        double* d = c->d_ad;
        auto take = [&](size_t k) {
            double* r = d;
            d += k;
            return r;
        };
        A.nb = take(P);
        A.tol = take(P);
        A.nrm = take(P);
        A.scale = take(P);
        A.H = take(Pm1 * m);
        A.cs = take(Pm);
        A.sn = take(Pm);
        A.g = take(Pm1);
        A.h1 = take(Pm1);
        A.h2 = take(Pm1);
        A.y = take(Pm);
        A.pack = take(4 * (size_t)P + 1);
        A.w = take(n3);
        A.st = c->d_adi;
        A.live = c->d_adi + kStWords;
        A.kd = c->d_adi + kStWords + P;
        ++g_graph_epoch;
    }
    const size_t red = (size_t)(m + 1) * P * B + 64;
    if (red > c->red_cap) {
        if (c->d_red) cudaFree(c->d_red);
        c->d_red = nullptr;
        c->red_cap = 0;
        if (dmalloc(&c->d_red, red) != cudaSuccess) return fail(c, SBIE_ERR_OOM, "reduction scratch");
        c->red_cap = red;
    }
    const size_t small = (size_t)(m + 1) * P + 64;
    if (2 * small > c->hred_cap) {
        if (c->h_red) cudaFreeHost(c->h_red);
        if (c->d_H) cudaFree(c->d_H);
        if (c->d_pvec) cudaFree(c->d_pvec);
        c->h_red = nullptr;
        c->d_H = c->d_pvec = nullptr;
        c->hred_cap = 0;
        if (cudaMallocHost(reinterpret_cast<void**>(&c->h_red), sizeof(double) * 2 * small) != cudaSuccess ||
            dmalloc(&c->d_H, small) != cudaSuccess || dmalloc(&c->d_pvec, small) != cudaSuccess)
            return fail(c, SBIE_ERR_OOM, "small solver buffers");
        c->hred_cap = 2 * small;
    }
    return SBIE_OK;
}

// Per-problem 2-norms of v (all problems of the system).
sbie_status seg_norms(const Sys& S, const double* v, std::vector<double>& out) {
    sbie_ctx* c = S.top;
    if (!c->d_pvec || !c->h_red || !c->d_red || c->hred_cap < 2 * (size_t)S.P)
        return fail(c, SBIE_ERR_ARG, "internal: solver buffers not allocated");
    CK(seg_dots(c, v, 1, S.n3, v, S.n3, c->d_seg3, S.P, c->d_pvec));
    CK(cudaMemcpyAsync(c->h_red, c->d_pvec, sizeof(double) * S.P, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out.resize(S.P);
    for (int p = 0; p < S.P; ++p) out[p] = std::sqrt(std::max(0.0, c->h_red[p]));
    return SBIE_OK;
}

// Stage a per-problem (or [k][P]) host array into the device matrix d_H.
sbie_status stage_H(sbie_ctx* c, const double* host, size_t count) {
    if (!c->h_red || !c->d_H || 2 * count > c->hred_cap) return fail(c, SBIE_ERR_ARG, "internal: staging overflow");
    double* st = c->h_red + c->hred_cap / 2;
    std::memcpy(st, host, sizeof(double) * count);
    CK(cudaMemcpyAsync(c->d_H, st, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
    return SBIE_OK;
}

struct GmresOut {
    int iters = 0, restarts = 0, graph_cycles = 0;
    std::vector<double> rel;  // per problem, residual of the final iterate recomputed with A
};

using AFn = std::function<sbie_status(const double*, double*)>;

// Kernel-launch counters of every context a system touches (top and parts).
std::vector<std::pair<sbie_ctx*, long long>> launch_counters(const Sys& S) {
    std::vector<std::pair<sbie_ctx*, long long>> v;
    v.push_back({S.top, S.top->n_launch});
    for (sbie_ctx* q : S.parts)
        if (q != S.top) v.push_back({q, q->n_launch});
    return v;
}

long long total_launches(const Sys& S) {
    long long t = 0;
    for (auto& pr : launch_counters(S)) t += pr.second;
    return t;
}

// One Arnoldi iteration of the device-resident cycle (krylov.cu): w = A V_k
// (A M^{-1} V_k with a right preconditioner), classical Gram-Schmidt twice,
// Givens update and convergence test per problem, V_{k+1} = w / ||w||.
sbie_status enqueue_iteration(const Sys& S, const AFn& A, const AFn* M, cudaGraphConditionalHandle cond,
                              bool has_cond) {
    sbie_ctx* c = S.top;
    const ArnoldiDev& AD = c->ad;
    CK(arnoldi_copy_k(c, AD, c->d_V, S.n3, c->d_vk));
    if (M) {
        CKS((*M)(c->d_vk, c->d_pz));
        CKS(A(c->d_pz, AD.w));
    } else {
        CKS(A(c->d_vk, AD.w));
    }
    StageScope sc(c, ST_BLAS);
    CK(arnoldi_orthogonalise(c, AD, c->d_V, S.n3, c->d_seg3, c->d_node_prob));
    CK(arnoldi_step_end(c, AD, c->d_V, S.n3, c->d_node_prob, cond, has_cond));
    return SBIE_OK;
}

// The restart cycle as a CUDA graph: one WHILE node whose body is one
// iteration; the advance kernel sets the condition.  Captured once per
// (operator, arithmetic, preconditioner) and reused while the device
// addresses and far-field tilings it holds are unchanged.
sbie_status cycle_graph(const Sys& S, const AFn& A, const AFn* M, int key, CycleGraph** out) {
    sbie_ctx* c = S.top;
    const unsigned long long ep = g_graph_epoch.load();
    for (size_t i = 0; i < c->graphs.size();) {
        CycleGraph& g = c->graphs[i];
        if (g.key == key && g.epoch == ep) {
            *out = &g;
            return SBIE_OK;
        }
        if (g.key == key || g.epoch != ep) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            c->graphs.erase(c->graphs.begin() + i);
        } else {
            ++i;
        }
    }
    CycleGraph g;
    g.key = key;
    g.epoch = ep;
    CK(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault);
    // the parameter union has no default constructor: zeroed raw storage
    alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
    std::memset(np_raw, 0, sizeof(np_raw));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np);
    sbie_status st = SBIE_OK;
    auto counters = launch_counters(S);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            st = enqueue_iteration(S, A, M, cond, true);
            cudaGraph_t captured = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &captured);
            if (e == cudaSuccess) e = e2;
        }
    }
    // the captured launches run once per iteration: count them when they do
    g.body_launches = 0;
    for (auto& pr : launch_counters(S)) g.body_launches += pr.second;
    for (auto& pr : counters) {
        g.body_launches -= pr.second;
        pr.first->n_launch = pr.second;
    }
    if (st == SBIE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (st != SBIE_OK || e != cudaSuccess) {
        cudaGraphDestroy(g.graph);
        cudaGetLastError();
        return fail(c, st != SBIE_OK ? st : SBIE_ERR_CUDA,
                    std::string("cycle graph: ") + (e != cudaSuccess ? cudaGetErrorString(e) : c->err));
    }
    c->graphs.push_back(g);
    *out = &c->graphs.back();
    return SBIE_OK;
}

// Restarted GMRES, one Krylov space per problem (classical Gram-Schmidt
// applied twice), x0 = 0.  Problem p runs while want[p] and its relative
// residual exceeds tol[p]; the residual is recomputed as b - A x at every
// restart.  Each restart cycle runs on the device (krylov.cu): as one graph
// launch when the context uses graphs and is not profiling, otherwise
// stepped from the host one iteration at a time.  `key` names the operator,
// arithmetic and preconditioner for the graph cache.  With trust_estimate the
// true residual is not recomputed after a cycle in which every problem
// stopped on its estimate (the caller forms its own residual next).
sbie_status gmres(const Sys& S, const AFn& A, const double* b, double* x, const std::vector<double>& tol,
                  const std::vector<char>& want, int restart, int max_iter, GmresOut& go, const AFn* M, int key,
                  bool trust_estimate = false) {
    sbie_ctx* c = S.top;
    const long long n3 = S.n3;
    const int P = S.P;
    restart = std::max(1, std::min(restart, 250));
    CKS(ensure_krylov(c, restart, P));
    if (c->ad.P != P) return fail(c, SBIE_ERR_ARG, "internal: cycle state sized for another system");
    const ArnoldiDev& AD = c->ad;
    const int m = restart;
    std::vector<double> nb, beta;
    CKS(seg_norms(S, b, nb));
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n3, c->stream));
    go = GmresOut();
    go.rel.assign(P, 0.0);
    for (int p = 0; p < P; ++p)
        if (!std::isfinite(nb[p])) return fail(c, SBIE_ERR_NUMERIC, "right-hand side is not finite");
    std::vector<char> active(P, 0);
    for (int p = 0; p < P; ++p) active[p] = want[p] && nb[p] > 0.0 && 1.0 > tol[p];
    double* r = c->d_res;
    CK(cudaMemcpyAsync(r, b, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
    beta = nb;
    std::vector<double> stage(P);
    bool graphs = c->opts.use_graphs != 0;
    int total = 0;
    auto any = [](const std::vector<char>& v) {
        for (char q : v)
            if (q) return true;
        return false;
    };
    while (any(active) && total < max_iter) {
        const int mm = std::min(m, max_iter - total);
        double* V = c->d_V;
        for (int p = 0; p < P; ++p) stage[p] = active[p] ? 1.0 / beta[p] : 0.0;
        CKS(stage_H(c, stage.data(), P));
        CK(seg_scale(c, r, c->d_H, c->d_node_prob, V, n3));
        for (int p = 0; p < P; ++p) {
            c->h_pack[p] = nb[p];
            c->h_pack[P + p] = tol[p];
            c->h_pack[2 * P + p] = beta[p];
            c->h_pack[3 * P + p] = active[p] ? 1.0 : 0.0;
        }
        c->h_pack[4 * P] = mm;
        CK(cudaMemcpyAsync(AD.pack, c->h_pack, sizeof(double) * (4 * (size_t)P + 1), cudaMemcpyHostToDevice, c->stream));
        CK(arnoldi_cycle_init(c, AD));
        // inside the cycle the far field skips problems that stopped
        {
            int off = 0;
            for (sbie_ctx* q : S.parts) {
                q->far_live = AD.live;
                q->far_live_off = off;
                off += q->n_prob;
            }
        }
        struct Unmask {
            const Sys& S;
            ~Unmask() {
                for (sbie_ctx* q : S.parts) q->far_live = nullptr;
            }
        } unmask{S};
        CycleGraph* g = nullptr;
        if (graphs && !c->prof.on) {
            if (cycle_graph(S, A, M, key, &g) == SBIE_OK) {
                CK(cudaGraphLaunch(g->exec, c->stream));
                ++go.graph_cycles;
            } else {
                graphs = false;  // host-stepped from here on; the reason stays in the context's error text
                g = nullptr;
            }
        }
        if (!g) {
            for (int it = 0; it < mm; ++it) {
                CKS(enqueue_iteration(S, A, M, cudaGraphConditionalHandle{}, false));
                if (c->prof.on) c->prof.arnoldi_vectors += 4LL * (it + 1) + 4;
                CK(cudaMemcpyAsync(c->h_st, AD.st, sizeof(int) * kStWords, cudaMemcpyDeviceToHost, c->stream));
                CK(cudaStreamSynchronize(c->stream));
                if (!c->h_st[2]) break;
            }
        }
        for (sbie_ctx* q : S.parts) q->far_live = nullptr;
        // x += V y (x += M^{-1} V y), then the true residual
        if (M) {
            double* t = c->d_pz + n3;
            CK(cudaMemsetAsync(t, 0, sizeof(double) * n3, c->stream));
            CK(arnoldi_finish(c, AD, V, n3, c->d_node_prob, t));
            CKS((*M)(t, c->d_pz));
            CK(blas_axpy(c, 1.0, c->d_pz, x, n3));
        } else {
            CK(arnoldi_finish(c, AD, V, n3, c->d_node_prob, x));
        }
        CK(cudaMemcpyAsync(c->h_st, AD.st, sizeof(int) * kStWords, cudaMemcpyDeviceToHost, c->stream));
        if (trust_estimate) {
            // every problem stopped on its Givens residual estimate: the
            // caller forms the residual itself, so the cycle's own b - A x is
            // not needed
            CK(cudaStreamSynchronize(c->stream));
            if (c->h_st[3]) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf in the Krylov basis");
            if (!c->h_st[4]) {
                const int kexec = c->h_st[0];
                if (g) c->n_launch += (long long)kexec * g->body_launches;
                total += kexec;
                ++go.restarts;
                for (int p = 0; p < P; ++p) beta[p] = active[p] ? tol[p] * nb[p] : beta[p];
                break;
            }
        }
        CKS(A(x, r));
        CK(blas_lincomb(c, 1.0, b, -1.0, r, r, n3));
        CKS(seg_norms(S, r, beta));  // synchronises the stream: h_st is current
        const int kexec = c->h_st[0];
        if (g) c->n_launch += (long long)kexec * g->body_launches;
        if (c->h_st[3]) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf in the Krylov basis");
        total += kexec;
        for (int p = 0; p < P; ++p) {
            if (!std::isfinite(beta[p])) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf residual");
            active[p] = want[p] && nb[p] > 0.0 && beta[p] / nb[p] > tol[p];
        }
        ++go.restarts;
        if (kexec == 0) break;
    }
    go.iters = total;
    for (int p = 0; p < P; ++p) go.rel[p] = nb[p] > 0.0 ? beta[p] / nb[p] : 0.0;
    return SBIE_OK;
}

// Solve A x = b to the FP64-accurate residual tolerance, every problem of the
// system at once.  SBIE_FP64 / SBIE_FP64_DF: GMRES on the FP64-accurate
// operator.  SBIE_MIXED: iterative refinement -- residuals b - A x with the
// FP64-accurate operator, corrections by GMRES on the FP32 operator.
sbie_status ensure_preconditioner(const Sys& S, int op);

// Bound on the FP32 operator's relative error (the mixed-precision apply
// parity bound) used to decide when a residual may be updated in FP32.
constexpr double kFp32OpErr = 2e-5;
// Smallest inner (FP32-operator) GMRES tolerance of a correction.  The first
// correction goes this deep, a little below the FP32 operator's own error, so
// that the second correction is small enough for its residual to be updated
// with the FP32 operator: a solve to 1e-8 then forms one FP64-accurate
// residual instead of two.
constexpr double kInnerTolMin = 1e-6;
// Largest inner tolerance: a later correction only has to take the residual
// from rel to half the tolerance (0.5 tol / rel), never less than a factor 10.
constexpr double kInnerTolMax = 0.1;

sbie_status solve_sys(const Sys& S, int op, const double* b, double* x, sbie_solve_info* info) {
    sbie_ctx* c = S.top;
    const long long n3 = S.n3;
    const int P = S.P;
    const int hm = hi_mode(c);
    AFn A64 = [&](const double* in, double* out) { return apply_sys(S, op, hm, in, out); };
    AFn A32 = [&](const double* in, double* out) { return apply_sys(S, op, kModeF32, in, out); };
    CKS(ensure_self_gemm(S));
    if (op == SBIE_OP_SQUIRMER) CKS(ensure_squirmer_buffers(S));
    CKS(ensure_preconditioner(S, op));
    const int slot = prec_slot(op);
    // the pair preconditioner belongs to the resistance and mobility operators
    bool prec = false;
    if (op == SBIE_OP_RESISTANCE || op == SBIE_OP_MOBILITY)
        for (sbie_ctx* q : S.parts) prec |= q->prec[slot].kind > 0;
    AFn Mf = [&](const double* in, double* out) {
        for (size_t i = 0; i < S.parts.size(); ++i) {
            sbie_ctx* q = S.parts[i];
            if (q->prec[slot].kind > 0) {
                StageScope st(q, ST_OTHER);
                cudaError_t e = precond_apply(q, slot, in + S.off3[i], out + S.off3[i], q->opts.prec == SBIE_MIXED);
                if (e != cudaSuccess) return fail(c, SBIE_ERR_CUDA, std::string("preconditioner: ") + cudaGetErrorString(e));
            } else {
                cudaError_t e = cudaMemcpyAsync(out + S.off3[i], in + S.off3[i], sizeof(double) * q->N * 3,
                                                cudaMemcpyDeviceToDevice, c->stream);
                if (e != cudaSuccess) return fail(c, SBIE_ERR_CUDA, cudaGetErrorString(e));
            }
        }
        return SBIE_OK;
    };
    const AFn* M = prec ? &Mf : nullptr;
    auto key_of = [&](int mode) { return (op * 4 + mode) * 2 + (prec ? 1 : 0); };
    if (prec && !c->d_pz && dmalloc(&c->d_pz, 2 * (size_t)n3) != cudaSuccess)
        return fail(c, SBIE_ERR_OOM, "preconditioner buffers");
    const double tol = c->opts.tol;
    GmresOut go;
    sbie_solve_info inf{};
    std::vector<double> rel(P, 0.0);
    // reduction and staging buffers must exist before the first norm
    CKS(ensure_krylov(c, std::max(1, std::min(c->opts.restart, 250)), P));
    if (c->opts.prec != SBIE_MIXED || op == kOpMagnetic) {
        CKS(gmres(S, A64, b, x, std::vector<double>(P, tol), std::vector<char>(P, 1), c->opts.restart,
                  c->opts.max_iter, go, M, key_of(hm)));
        inf.iters = go.iters;
        inf.restarts = go.restarts;
        inf.graph_cycles = go.graph_cycles;
        rel = go.rel;
    } else {
        std::vector<double> nb;
        CKS(seg_norms(S, b, nb));
        CK(cudaMemsetAsync(x, 0, sizeof(double) * n3, c->stream));
        double* r = c->d_tmp2;
        double* d = c->d_tmp;
        CK(cudaMemcpyAsync(r, b, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c->stream));
        for (int p = 0; p < P; ++p) rel[p] = nb[p] > 0 ? 1.0 : 0.0;
        int iters = 0, outers = 0;
        double eps32 = kFp32OpErr;
        auto worst = [&]() { return *std::max_element(rel.begin(), rel.end()); };
        while (worst() > tol && iters < c->opts.max_iter && outers < 20) {
            std::vector<double> itol(P);
            std::vector<char> want(P);
            for (int p = 0; p < P; ++p) {
                want[p] = rel[p] > tol;
                itol[p] = std::min(kInnerTolMax, std::max(kInnerTolMin, 0.5 * tol / std::max(rel[p], 1e-300)));
            }
            CKS(gmres(S, A32, r, d, itol, want, c->opts.restart, c->opts.max_iter - iters, go, M, key_of(kModeF32),
                      true));
            iters += go.iters;
            inf.restarts += go.restarts;
            inf.graph_cycles += go.graph_cycles;
            CK(blas_axpy(c, 1.0, d, x, n3));
            // New residual.  After the first correction it is r - A d by
            // linearity, and A d may use the FP32 operator when the
            // correction is small: the error of that update is about
            // eps32 ||d|| / ||x|| relative to ||b||, with eps32 the FP32
            // operator's relative error, and it is kept below a tenth of the
            // tolerance.  eps32 is measured on this system at the first
            // FP64-accurate residual (A x in both arithmetics) and taken ten
            // times over, never below 1e-6; otherwise the bound 2e-5 of the
            // mixed-precision apply holds.  Else r = b - A x with the
            // FP64-accurate operator.
            double* t = c->d_out;  // not used by the solve's callers until it returns
            bool cheap = outers > 0;
            if (cheap) {
                std::vector<double> dn, xn;
                CKS(seg_norms(S, d, dn));
                CKS(seg_norms(S, x, xn));
                inf.last_correction = 0.0;
                for (int p = 0; p < P; ++p) {
                    if (xn[p] > 0.0) inf.last_correction = std::max(inf.last_correction, dn[p] / xn[p]);
                    if (dn[p] > 0.0 && !(eps32 * dn[p] <= 0.1 * tol * xn[p])) cheap = false;
                }
            }
            if (cheap) {
                CKS(A32(d, t));
                CK(blas_axpy(c, -1.0, t, r, n3));
                ++inf.fp32_residual_updates;
            } else {
                CKS(A64(x, r));
                CK(blas_lincomb(c, 1.0, b, -1.0, r, r, n3));
                if (outers == 0) {  // eps32 from A x: d <- A64 x - A32 x (d is free until the next GMRES)
                    CKS(A32(x, t));
                    CK(blas_lincomb(c, 1.0, b, -1.0, r, d, n3));
                    std::vector<double> an, en;
                    CKS(seg_norms(S, d, an));
                    CK(blas_axpy(c, -1.0, t, d, n3));
                    CKS(seg_norms(S, d, en));
                    double worst = 0.0;
                    for (int p = 0; p < P; ++p)
                        if (an[p] > 0.0) worst = std::max(worst, en[p] / an[p]);
                    if (std::isfinite(worst)) eps32 = std::min(kFp32OpErr, std::max(1e-6, 10.0 * worst));
                    inf.fp32_op_err = worst;
                }
            }
            std::vector<double> rn;
            CKS(seg_norms(S, r, rn));
            for (int p = 0; p < P; ++p) {
                if (!std::isfinite(rn[p])) return fail(c, SBIE_ERR_NUMERIC, "NaN/Inf residual");
                rel[p] = nb[p] > 0 ? rn[p] / nb[p] : 0.0;
            }
            ++outers;
            if (go.iters == 0) break;
        }
        inf.iters = iters;
        inf.refinements = outers;
    }
    CKS(check_self_gemm(S));
    inf.rel_residual_true = *std::max_element(rel.begin(), rel.end());
    long long nn = 0;
    for (sbie_ctx* q : S.parts) nn += q->n_near;
    inf.n_near_pairs = nn;
    if (info) *info = inf;
    return inf.rel_residual_true <= tol ? SBIE_OK : SBIE_ERR_NOT_CONVERGED;
}

bool finite_all(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

sbie_status check_opts(const sbie_opts* opts) {
    if (opts->p < 1 || opts->p > kMaxP) return fail(nullptr, SBIE_ERR_ARG, "p must be in [1, 24]");
    if (!(opts->eta >= 0.0) || !std::isfinite(opts->eta)) return fail(nullptr, SBIE_ERR_ARG, "eta must be >= 0");
    if (opts->prec != SBIE_FP64 && opts->prec != SBIE_MIXED && opts->prec != SBIE_FP64_DF)
        return fail(nullptr, SBIE_ERR_ARG, "bad precision");
    if (opts->mem_kind != 0 && opts->mem_kind != 1) return fail(nullptr, SBIE_ERR_ARG, "mem_kind must be 0 or 1");
    if (opts->use_learned_precond < 0 || opts->use_learned_precond > 2)
        return fail(nullptr, SBIE_ERR_ARG, "use_learned_precond must be 0, 1 or 2");
    if (opts->use_learned_precond == 1 && !opts->mlp_weights_path)
        return fail(nullptr, SBIE_ERR_ARG, "the learned preconditioner needs mlp_weights_path");
    if (!(opts->tol > 0.0) || opts->restart < 1 || opts->max_iter < 0)
        return fail(nullptr, SBIE_ERR_ARG, "need tol > 0, restart >= 1, max_iter >= 0");
    if (opts->use_graphs != 0 && opts->use_graphs != 1) return fail(nullptr, SBIE_ERR_ARG, "use_graphs must be 0 or 1");
    if (opts->near_scheme != 0 && opts->near_scheme != 1)
        return fail(nullptr, SBIE_ERR_ARG, "near_scheme must be 0 or 1");
    return SBIE_OK;
}

// One context for spheres of one VSH order p = o.p, holding the independent
// problems prob_sph[q] .. prob_sph[q+1]-1.  Close pairs never cross problems.
sbie_status create_part(const sbie_opts& o, int n, const double* centres, const double* radii,
                        const std::vector<int>& prob_sph, cudaStream_t stream, sbie_ctx** out) {
    sbie_ctx* c = new (std::nothrow) sbie_ctx();
    if (!c) return fail(nullptr, SBIE_ERR_OOM, "host allocation");
    c->opts = o;
    c->n = n;
    c->p = o.p;
    c->nlat = c->p + 1;
    c->nlon = 2 * c->p + 2;
    c->npn = c->nlat * c->nlon;
    c->N = (long long)n * c->npn;
    c->h_c.assign(centres, centres + 3 * (size_t)n);
    c->h_a.assign(radii, radii + n);
    c->n_prob = (int)prob_sph.size() - 1;
    c->h_prob_sph = prob_sph;
    std::vector<int> sph_prob(n);
    for (int q = 0; q < c->n_prob; ++q)
        for (int i = prob_sph[q]; i < prob_sph[q + 1]; ++i) sph_prob[i] = q;
    // close pairs (negation of Eq. 4.5) and overlap check, within each problem
    c->h_near_ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const int q = sph_prob[i];
        for (int k = prob_sph[q]; k < prob_sph[q + 1]; ++k) {
            if (k == i) continue;
            double dx = centres[3 * i] - centres[3 * k], dy = centres[3 * i + 1] - centres[3 * k + 1],
                   dz = centres[3 * i + 2] - centres[3 * k + 2];
            double gap = std::sqrt(dx * dx + dy * dy + dz * dz) - radii[i] - radii[k];
            if (gap <= 0.0) {
                g_last_error = "spheres " + std::to_string(i) + " and " + std::to_string(k) + " overlap or touch";
                delete c;
                return SBIE_ERR_OVERLAP;
            }
            if (gap < o.eta * 2.0 * std::max(radii[i], radii[k])) c->h_near_idx.push_back(k);
        }
        c->h_near_ptr[i + 1] = (int)c->h_near_idx.size();
    }
    c->n_near = (long long)c->h_near_idx.size();
    c->far_pair_count = far_pairs(c);
    c->seg3.resize(c->n_prob + 1);
    for (int q = 0; q <= c->n_prob; ++q) c->seg3[q] = (long long)prob_sph[q] * c->npn * 3;
    std::vector<int> node_prob((size_t)c->N);
    for (long long i = 0; i < c->N; ++i) node_prob[i] = sph_prob[i / c->npn];

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
    if (stream || o.stream) {
        c->stream = stream ? stream : (cudaStream_t)o.stream;
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
    ok &= dmalloc(&c->d_prob_sph, (size_t)c->n_prob + 1) == cudaSuccess;
    ok &= dmalloc(&c->d_sph_prob, (size_t)n) == cudaSuccess;
    ok &= dmalloc(&c->d_node_prob, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_seg3, (size_t)c->n_prob + 1) == cudaSuccess;
    ok &= dmalloc(&c->d_tab, (size_t)c->tl.total) == cudaSuccess;
    ok &= dmalloc(&c->d_coef, (size_t)n * 3 * P1 * P1 * 2) == cudaSuccess;
    if (c->n_near > 0) {
        ok &= dmalloc(&c->d_chan, (size_t)n * Kc * kTracChannels) == cudaSuccess;
        ok &= dmalloc(&c->d_chanf, (size_t)n * Kc * 28) == cudaSuccess;
    }
    ok &= dmalloc(&c->d_mom, 6 * (size_t)n) == cudaSuccess;
    ok &= dmalloc(&c->d_src64, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_srcf, (size_t)N) == cudaSuccess;
    for (double** p : {&c->d_in, &c->d_out, &c->d_tmp, &c->d_tmp2, &c->d_xsol, &c->d_rhs, &c->d_res})
        ok &= dmalloc(p, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&c->d_small, 3 * (size_t)n * 6 + 32) == cudaSuccess;
    if (!ok) return bail(SBIE_ERR_OOM, "device allocation failed");
    choose_tuning(c);
    {
        sbie_status s = ensure_part(c);
        if (s != SBIE_OK) return bail(s, c->err);
    }
    e = h2d(c->stream, c->d_c, centres, 3 * (size_t)n);
    if (e == cudaSuccess) e = h2d(c->stream, c->d_a, radii, (size_t)n);
    if (e == cudaSuccess) e = h2d(c->stream, c->d_near_ptr, c->h_near_ptr.data(), (size_t)n + 1);
    if (e == cudaSuccess && c->n_near > 0)
        e = h2d(c->stream, c->d_near_idx, c->h_near_idx.data(), (size_t)c->n_near);
    if (e == cudaSuccess)
        e = h2d(c->stream, c->d_prob_sph, prob_sph.data(), (size_t)c->n_prob + 1);
    if (e == cudaSuccess) e = h2d(c->stream, c->d_sph_prob, sph_prob.data(), (size_t)n);
    if (e == cudaSuccess) e = h2d(c->stream, c->d_node_prob, node_prob.data(), (size_t)N);
    if (e == cudaSuccess)
        e = h2d(c->stream, c->d_seg3, c->seg3.data(), c->seg3.size());
    if (e == cudaSuccess) e = h2d(c->stream, c->d_tab, htab.data(), htab.size());
    if (e == cudaSuccess) e = launch_geometry(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    if (o.near_scheme == 1 && c->n_near > 0) {
        sbie_status s2 = setup_near_fft(c, htab);
        if (s2 != SBIE_OK) return bail(s2, c->err);
    }
    c->err = "no error";
    *out = c;
    return SBIE_OK;
}

// Copy a user array (host or device per opts.mem_kind) into internal order on
// the device: per node (3 doubles each) if nodal, else per sphere.
sbie_status to_internal(sbie_ctx* c, const double* user, double* dev, bool nodal) {
    const cudaMemcpyKind kind = c->opts.mem_kind == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (!c->is_batch) {
        const size_t cnt = nodal ? (size_t)c->N : (size_t)c->n;
        if (user != dev) CK(cudaMemcpyAsync(dev, user, sizeof(double) * 3 * cnt, kind, c->stream));
        return SBIE_OK;
    }
    long long sph_base[64] = {0};
    for (size_t s = 1; s < c->parts.size() && s < 64; ++s) sph_base[s] = sph_base[s - 1] + c->parts[s - 1]->n;
    for (int q = 0; q < c->n_prob; ++q) {
        const int s = c->prob_part[q];
        sbie_ctx* part = c->parts[s];
        const long long isph = sph_base[s] + part->h_prob_sph[c->prob_local[q]];
        long long ioff, uoff, cnt;
        if (nodal) {
            ioff = c->part_off3[s] / 3 + (long long)part->h_prob_sph[c->prob_local[q]] * part->npn;
            uoff = c->prob_user_node[q];
            cnt = c->prob_user_node[q + 1] - uoff;
        } else {
            ioff = isph;
            uoff = c->prob_user_sph[q];
            cnt = c->prob_user_sph[q + 1] - uoff;
        }
        CK(cudaMemcpyAsync(dev + 3 * ioff, user + 3 * uoff, sizeof(double) * 3 * cnt, kind, c->stream));
    }
    return SBIE_OK;
}

sbie_status to_user(sbie_ctx* c, const double* dev, double* user, bool nodal) {
    const cudaMemcpyKind kind = c->opts.mem_kind == 0 ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (!c->is_batch) {
        const size_t cnt = nodal ? (size_t)c->N : (size_t)c->n;
        if (user != dev) CK(cudaMemcpyAsync(user, dev, sizeof(double) * 3 * cnt, kind, c->stream));
        return SBIE_OK;
    }
    long long sph_base[64] = {0};
    for (size_t s = 1; s < c->parts.size() && s < 64; ++s) sph_base[s] = sph_base[s - 1] + c->parts[s - 1]->n;
    for (int q = 0; q < c->n_prob; ++q) {
        const int s = c->prob_part[q];
        sbie_ctx* part = c->parts[s];
        long long ioff, uoff, cnt;
        if (nodal) {
            ioff = c->part_off3[s] / 3 + (long long)part->h_prob_sph[c->prob_local[q]] * part->npn;
            uoff = c->prob_user_node[q];
            cnt = c->prob_user_node[q + 1] - uoff;
        } else {
            ioff = sph_base[s] + part->h_prob_sph[c->prob_local[q]];
            uoff = c->prob_user_sph[q];
            cnt = c->prob_user_sph[q + 1] - uoff;
        }
        CK(cudaMemcpyAsync(user + 3 * uoff, dev + 3 * ioff, sizeof(double) * 3 * cnt, kind, c->stream));
    }
    return SBIE_OK;
}

// ---- pair preconditioner and pair network (kernels in precond.cu, mlp.cu)

struct PairNet {
    int op = SBIE_OP_RESISTANCE;        // operator whose blocks it predicts
    std::vector<float> params;          // FP32 weights (mlp_layout)
    float in_mean[kMlpIn], in_std[kMlpIn];
    float in_min[kMlpIn], in_max[kMlpIn];  // range of the training inputs
    std::vector<float> out_mean, out_std;
    int p_train = 0;
    // true when x lies inside the trained input range (a pair outside it is
    // left out of the preconditioner rather than extrapolated)
    bool covers(const float* x) const {
        for (int j = 0; j < kMlpIn; ++j) {
            const float slack = 1e-4f * (1.f + std::fabs(in_min[j]) + std::fabs(in_max[j]));
            if (!(x[j] >= in_min[j] - slack && x[j] <= in_max[j] + slack)) return false;
        }
        return true;
    }
};

}  // namespace
// the networks of one weights file, at most one per operator
struct sbie::PairNetSet {
    std::vector<PairNet> nets;
    const PairNet* for_op(int op) const {
        for (const PairNet& n : nets)
            if (n.op == op) return &n;
        return nullptr;
    }
};
namespace {

// File: magic "SBIEPN03", int count, then per network int[7] {L, in, hidden,
// out, p of the probed grid, parameter count, operator}, input mean, std,
// min, max, output mean, std, parameters (all float).
const char kNetMagic[9] = "SBIEPN03";

sbie_status net_save(const char* path, const PairNetSet& set) {
    std::ofstream f(path, std::ios::binary);
    if (!f) return fail(nullptr, SBIE_ERR_ARG, std::string("cannot write ") + path);
    f.write(kNetMagic, 8);
    const int count = (int)set.nets.size();
    f.write(reinterpret_cast<const char*>(&count), sizeof(count));
    for (const PairNet& net : set.nets) {
        int hdr[7] = {kPrecL, kMlpIn, kMlpHidden, kMlpOut, net.p_train, (int)net.params.size(), net.op};
        f.write(reinterpret_cast<const char*>(hdr), sizeof(hdr));
        f.write(reinterpret_cast<const char*>(net.in_mean), sizeof(net.in_mean));
        f.write(reinterpret_cast<const char*>(net.in_std), sizeof(net.in_std));
        f.write(reinterpret_cast<const char*>(net.in_min), sizeof(net.in_min));
        f.write(reinterpret_cast<const char*>(net.in_max), sizeof(net.in_max));
        f.write(reinterpret_cast<const char*>(net.out_mean.data()), sizeof(float) * kMlpOut);
        f.write(reinterpret_cast<const char*>(net.out_std.data()), sizeof(float) * kMlpOut);
        f.write(reinterpret_cast<const char*>(net.params.data()), sizeof(float) * net.params.size());
    }
    return f ? SBIE_OK : fail(nullptr, SBIE_ERR_ARG, "write failed");
}

sbie_status net_load(const char* path, PairNetSet& set) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(nullptr, SBIE_ERR_ARG, std::string("cannot read ") + path);
    char magic[8];
    int count = 0;
    f.read(magic, 8);
    f.read(reinterpret_cast<char*>(&count), sizeof(count));
    if (!f || std::memcmp(magic, kNetMagic, 8) != 0 || count < 1 || count > 2)
        return fail(nullptr, SBIE_ERR_ARG, std::string("not a pair-network file: ") + path);
    MlpLayout L = mlp_layout();
    set.nets.assign(count, PairNet());
    for (PairNet& net : set.nets) {
        int hdr[7];
        f.read(reinterpret_cast<char*>(hdr), sizeof(hdr));
        if (!f || hdr[0] != kPrecL || hdr[1] != kMlpIn || hdr[2] != kMlpHidden || hdr[3] != kMlpOut ||
            hdr[5] != (int)L.total || (hdr[6] != SBIE_OP_RESISTANCE && hdr[6] != SBIE_OP_MOBILITY))
            return fail(nullptr, SBIE_ERR_ARG, std::string("not a pair-network file: ") + path);
        net.p_train = hdr[4];
        net.op = hdr[6];
        net.out_mean.resize(kMlpOut);
        net.out_std.resize(kMlpOut);
        net.params.resize(L.total);
        f.read(reinterpret_cast<char*>(net.in_mean), sizeof(net.in_mean));
        f.read(reinterpret_cast<char*>(net.in_std), sizeof(net.in_std));
        f.read(reinterpret_cast<char*>(net.in_min), sizeof(net.in_min));
        f.read(reinterpret_cast<char*>(net.in_max), sizeof(net.in_max));
        f.read(reinterpret_cast<char*>(net.out_mean.data()), sizeof(float) * kMlpOut);
        f.read(reinterpret_cast<char*>(net.out_std.data()), sizeof(float) * kMlpOut);
        f.read(reinterpret_cast<char*>(net.params.data()), sizeof(float) * L.total);
    }
    return f ? SBIE_OK : fail(nullptr, SBIE_ERR_ARG, std::string("truncated pair-network file: ") + path);
}

// Exact low-mode blocks by probing context `c` (problems of sph_per_prob
// spheres): for each side s < nsides the 73 low modes are placed on local
// sphere s of every problem and operator `op` (resistance or mobility)
// applied in FP64; the low-mode analysis of every sphere's response fills
// out[s][sphere][row][mode] (host).
sbie_status probe_blocks(sbie_ctx* c, int op, int sph_per_prob, int nsides, std::vector<double>& out,
                         int mode = kModeF64) {
    std::vector<double> ZS, ZA;
    lowmode_tables(c->p, ZS, ZA);
    double *dZS = nullptr, *dZA = nullptr, *dB = nullptr;
    const size_t per = (size_t)c->n * kLowModes * kLowModes;
    sbie_status st = SBIE_OK;
    if (dmalloc(&dZS, ZS.size()) != cudaSuccess || dmalloc(&dZA, ZA.size()) != cudaSuccess ||
        dmalloc(&dB, per * nsides) != cudaSuccess) {
        st = fail(c, SBIE_ERR_OOM, "probe buffers");
    }
    cudaError_t e = cudaSuccess;
    if (st == SBIE_OK) {
        e = h2d(c->stream, dZS, ZS.data(), ZS.size());
        if (e == cudaSuccess) e = h2d(c->stream, dZA, ZA.data(), ZA.size());
        for (int s = 0; s < nsides && e == cudaSuccess && st == SBIE_OK; ++s)
            for (int b = 0; b < kLowModes && e == cudaSuccess && st == SBIE_OK; ++b) {
                e = launch_probe_density(c, sph_per_prob, s, b, dZS, c->d_in);
                if (e == cudaSuccess) st = apply_dev(c, op, mode, c->d_in, c->d_out);
                if (st == SBIE_OK && e == cudaSuccess) e = launch_probe_analysis(c, dZA, c->d_out, b, dB + s * per);
            }
        if (e == cudaSuccess && st == SBIE_OK) {
            out.resize(per * nsides);
            e = d2h(c->stream, out.data(), dB, out.size());
        }
        if (e != cudaSuccess) st = fail(c, SBIE_ERR_CUDA, std::string("probe: ") + cudaGetErrorString(e));
    }
    for (double* p : {dZS, dZA, dB})
        if (p) cudaFree(p);
    return st;
}

sbie_status create_part(const sbie_opts& o, int n, const double* centres, const double* radii,
                        const std::vector<int>& prob_sph, cudaStream_t stream, sbie_ctx** out);

// Exact aligned blocks: source sphere (radius a_s) at the origin, target
// (radius a_t) at (0, 0, d); out [n][73][73] (target <- source).
sbie_status aligned_blocks(int n, const double* d, const double* a_s, const double* a_t, int p, double eta, int op,
                           std::vector<double>& out, int mode = kModeF64) {
    std::vector<double> cc((size_t)n * 6, 0.0), aa((size_t)n * 2);
    std::vector<int> ps(n + 1);
    for (int q = 0; q < n; ++q) {
        cc[6 * q + 5] = d[q];
        aa[2 * q] = a_s[q];
        aa[2 * q + 1] = a_t[q];
        ps[q] = 2 * q;
    }
    ps[n] = 2 * n;
    sbie_opts o;
    sphere_bie_default_opts(&o);
    o.p = p;
    o.eta = eta;
    sbie_ctx* pc = nullptr;
    CKS(create_part(o, 2 * n, cc.data(), aa.data(), ps, nullptr, &pc));
    std::vector<double> B;
    sbie_status st = probe_blocks(pc, op, 2, 1, B, mode);
    if (st == SBIE_OK) {
        out.resize((size_t)n * kLowModes * kLowModes);
        const size_t blk = (size_t)kLowModes * kLowModes;
        for (int q = 0; q < n; ++q) std::memcpy(out.data() + q * blk, B.data() + (2 * q + 1) * blk, sizeof(double) * blk);
    } else {
        g_last_error = pc->err;
    }
    free_all(pc);
    delete pc;
    return st;
}

// f(begin, end) over [0, n) split across the host's cores.
template <typename F>
void parallel_for(int n, F f) {
    const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int nt = std::max(1, std::min(hw, n / 16));
    if (nt == 1) {
        f(0, n);
        return;
    }
    std::vector<std::thread> th;
    for (int i = 0; i < nt; ++i) th.emplace_back(f, (int)((long long)n * i / nt), (int)((long long)n * (i + 1) / nt));
    for (auto& t : th) t.join();
}

void pair_frame(const double* cs, const double* ct, double Q[9], double* dist) {
    double u[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
    double d = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (double& v : u) v /= d;
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (std::fabs(u[a]) < std::fabs(u[ax])) ax = a;
    double e1[3] = {0, 0, 0};
    e1[ax] = 1.0;
    double dot = e1[0] * u[0] + e1[1] * u[1] + e1[2] * u[2];
    for (int a = 0; a < 3; ++a) e1[a] -= dot * u[a];
    double nn = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (double& v : e1) v /= nn;
    double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
    for (int a = 0; a < 3; ++a) {
        Q[3 * a + 0] = e1[a];
        Q[3 * a + 1] = e2[a];
        Q[3 * a + 2] = u[a];
    }
    *dist = d;
}

// Network blocks (pair frame, de-standardised) for inputs (0, 0, d, a_s, a_t).
// The network's standardised outputs for inputs X5 ([n][5]) on stream s into
// dY ([n][5329], device).
sbie_status net_forward_dev(const PairNet& net, const std::vector<float>& X5, cudaStream_t s, float* dY) {
    const int n = (int)(X5.size() / kMlpIn);
    MlpLayout L = mlp_layout();
    float *dw = nullptr, *dX = nullptr;
    __nv_bfloat16* dwb = nullptr;
    std::vector<float> Xs(X5.size());
    for (int q = 0; q < n; ++q)
        for (int j = 0; j < kMlpIn; ++j) Xs[q * kMlpIn + j] = (X5[q * kMlpIn + j] - net.in_mean[j]) / net.in_std[j];
    cudaError_t e = cudaMalloc(&dw, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&dwb, sizeof(__nv_bfloat16) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&dX, sizeof(float) * Xs.size());
    if (e == cudaSuccess) e = h2d(s, dw, net.params.data(), (size_t)L.total);
    if (e == cudaSuccess) e = h2d(s, dX, Xs.data(), Xs.size());
    if (e == cudaSuccess) e = mlp_to_bf16(s, dw, dwb);
    if (e == cudaSuccess) e = mlp_forward_dev(s, dw, dwb, n, dX, dY);
    for (void* p : {(void*)dw, (void*)dwb, (void*)dX})
        if (p) cudaFree(p);
    if (e != cudaSuccess) return fail(nullptr, SBIE_ERR_CUDA, std::string("network: ") + cudaGetErrorString(e));
    return SBIE_OK;
}

// The network's blocks for inputs X5, de-standardised, on the host.
sbie_status net_blocks(const PairNet& net, const std::vector<float>& X5, std::vector<double>& out) {
    const int n = (int)(X5.size() / kMlpIn);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(nullptr, SBIE_ERR_CUDA, "stream");
    float* dY = nullptr;
    std::vector<float> Y((size_t)n * kMlpOut);
    sbie_status st = SBIE_OK;
    if (cudaMalloc(&dY, sizeof(float) * Y.size()) != cudaSuccess) st = fail(nullptr, SBIE_ERR_OOM, "network outputs");
    if (st == SBIE_OK) st = net_forward_dev(net, X5, s, dY);
    if (st == SBIE_OK && d2h(s, Y.data(), dY, Y.size()) != cudaSuccess) st = fail(nullptr, SBIE_ERR_CUDA, "network outputs");
    if (dY) cudaFree(dY);
    cudaStreamDestroy(s);
    if (st != SBIE_OK) return st;
    out.resize(Y.size());
    for (size_t i = 0; i < Y.size(); ++i)
        out[i] = (double)Y[i] * net.out_std[i % kMlpOut] + net.out_mean[i % kMlpOut];
    return SBIE_OK;
}

sbie_status precond_setup(sbie_ctx* c, int op, int kind, const PairNet* net);

// The pair preconditioner of operator `op` for every part of a system, built
// at the first solve with that operator.  With the network (kind 1) and no
// network for `op` in the weights file, the solve runs unpreconditioned.
sbie_status ensure_preconditioner(const Sys& S, int op) {
    sbie_ctx* top = S.top;
    const int kind = top->opts.use_learned_precond, slot = prec_slot(op);
    if (kind == 0 || (op != SBIE_OP_RESISTANCE && op != SBIE_OP_MOBILITY)) return SBIE_OK;
    const PairNet* net = nullptr;
    if (kind == 1) {
        net = top->nets ? top->nets->for_op(op) : nullptr;
        if (!net) {
            for (sbie_ctx* q : S.parts) q->prec[slot].built = true;  // kind stays 0: no preconditioner
            return SBIE_OK;
        }
    }
    for (sbie_ctx* q : S.parts) {
        if (q->prec[slot].built) continue;
        sbie_status st = precond_setup(q, op, kind, net);
        if (st != SBIE_OK) {
            if (q != top) top->err = q->err;
            return st;
        }
    }
    return SBIE_OK;
}

// Exact pair-frame blocks of operator `op` for two-sphere configurations with
// gaps log-uniform in [gap_min, gap_max] (probing the close-pair path of the
// operator on the GPU), then the network trained on them with the library's
// own kernels; the last val_frac of the samples are held out.
sbie_status train_one(const sbie_pair_train_opts& o, int op, PairNet& net, sbie_pair_train_info& info) {
    auto t0 = std::chrono::steady_clock::now();
    const int n = o.n_samples;
    std::mt19937_64 rng(o.seed);
    std::uniform_real_distribution<double> U(std::log(o.gap_min), std::log(o.gap_max));
    std::vector<double> d(n), as(n, o.radius), at(n, o.radius);
    const bool ranged = o.radius_max > o.radius;
    std::uniform_real_distribution<double> R(o.radius, ranged ? o.radius_max : o.radius);
    for (int q = 0; q < n; ++q) {
        if (ranged) {
            as[q] = R(rng);
            at[q] = R(rng);
        }
        d[q] = as[q] + at[q] + std::exp(U(rng));
    }
    std::vector<double> blocks((size_t)n * kMlpOut);
    const int chunk = 4096;
    for (int q0 = 0; q0 < n; q0 += chunk) {
        const int m = std::min(chunk, n - q0);
        std::vector<double> out;
        // the FP32 operator: blocks to about 1e-6, far below the network's error
        CKS(aligned_blocks(m, d.data() + q0, as.data() + q0, at.data() + q0, o.p, 1e9, op, out, kModeF32));
        std::memcpy(blocks.data() + (size_t)q0 * kMlpOut, out.data(), sizeof(double) * out.size());
    }
    auto t1 = std::chrono::steady_clock::now();
    net = PairNet();
    net.op = op;
    net.p_train = o.p;
    std::vector<float> X((size_t)n * kMlpIn, 0.f);
    for (int q = 0; q < n; ++q) {
        X[q * kMlpIn + 2] = (float)d[q];
        X[q * kMlpIn + 3] = (float)as[q];
        X[q * kMlpIn + 4] = (float)at[q];
    }
    for (int j = 0; j < kMlpIn; ++j) {
        double s = 0, s2 = 0;
        for (int q = 0; q < n; ++q) {
            s += X[q * kMlpIn + j];
            s2 += (double)X[q * kMlpIn + j] * X[q * kMlpIn + j];
        }
        const double mu = s / n, var = std::max(0.0, s2 / n - mu * mu);
        net.in_min[j] = net.in_max[j] = X[j];
        for (int q = 0; q < n; ++q) {
            net.in_min[j] = std::min(net.in_min[j], X[q * kMlpIn + j]);
            net.in_max[j] = std::max(net.in_max[j], X[q * kMlpIn + j]);
        }
        net.in_mean[j] = (float)mu;
        net.in_std[j] = var > 1e-20 ? (float)std::sqrt(var) : 1.f;
    }
    net.out_mean.assign(kMlpOut, 0.f);
    net.out_std.assign(kMlpOut, 1.f);
    double smax = 0.0;
    std::vector<double> sd(kMlpOut);
    for (int k = 0; k < kMlpOut; ++k) {
        double s = 0, s2 = 0;
        for (int q = 0; q < n; ++q) {
            const double v = blocks[(size_t)q * kMlpOut + k];
            s += v;
            s2 += v * v;
        }
        const double mu = s / n;
        sd[k] = std::sqrt(std::max(0.0, s2 / n - mu * mu));
        net.out_mean[k] = (float)mu;
        smax = std::max(smax, sd[k]);
    }
    // Entries that do not vary over the samples (most of the block: in the
    // pair frame only modes of equal order m couple) get std 0, so that the
    // prediction is their mean exactly and the network's error there is not
    // added to the block; their standardised target is 0.
    for (int k = 0; k < kMlpOut; ++k) net.out_std[k] = sd[k] > 1e-6 * smax ? (float)sd[k] : 0.f;
    std::vector<float> Xs(X.size()), Ys((size_t)n * kMlpOut);
    for (int q = 0; q < n; ++q) {
        for (int j = 0; j < kMlpIn; ++j) Xs[q * kMlpIn + j] = (X[q * kMlpIn + j] - net.in_mean[j]) / net.in_std[j];
        for (int k = 0; k < kMlpOut; ++k)
            Ys[(size_t)q * kMlpOut + k] =
                net.out_std[k] > 0.f
                    ? (float)((blocks[(size_t)q * kMlpOut + k] - net.out_mean[k]) / net.out_std[k])
                    : 0.f;
    }
    const int nval = (int)(o.val_frac * n), ntr = n - nval;
    mlp_init(o.seed + 1, net.params);
    MlpTrainOpts to;
    to.epochs = o.epochs;
    to.batch = o.batch;
    to.lr = o.lr;
    to.seed = o.seed + 2;
    std::vector<double> hist;
    cudaError_t e = mlp_train(to, ntr, Xs.data(), Ys.data(), net.params.data(), hist);
    if (e != cudaSuccess) return fail(nullptr, SBIE_ERR_CUDA, std::string("training: ") + cudaGetErrorString(e));
    auto t2 = std::chrono::steady_clock::now();
    double val = 0.0;
    if (nval > 0) {
        std::vector<float> Xv(X.begin() + (size_t)ntr * kMlpIn, X.end());
        std::vector<double> P;
        CKS(net_blocks(net, Xv, P));
        for (int q = 0; q < nval; ++q) {
            double num = 0, den = 0;
            for (int k = 0; k < kMlpOut; ++k) {
                const double t = blocks[(size_t)(ntr + q) * kMlpOut + k], y = P[(size_t)q * kMlpOut + k];
                num += (y - t) * (y - t);
                den += t * t;
            }
            val += std::sqrt(num / den);
        }
        val /= nval;
    }
    info.train_loss = hist.empty() ? 0.0 : hist.back();
    info.val_rel_err = val;
    info.t_data_s = std::chrono::duration<double>(t1 - t0).count();
    info.t_train_s = std::chrono::duration<double>(t2 - t1).count();
    info.n_train = ntr;
    info.n_val = nval;
    return SBIE_OK;
}

// Builds the pair preconditioner of operator `op` on one part (kind 1:
// network, 2: exact blocks).
// Own low-mode blocks of operator `op` (single-sphere problems): L_i depends
// on the sphere's radius only, so each distinct radius is probed once, G of
// its 73 low modes per pass on G copies of the sphere (each its own problem),
// as many passes as needed.  Lu [distinct radii][73][73], uid[i] = the block
// of sphere i.
sbie_status own_blocks(sbie_ctx* c, const sbie_opts& o, int op, std::vector<double>& Lu, std::vector<int>& uid) {
    const int n = c->n, NM = kLowModes;
    const size_t blk = (size_t)NM * NM;
    std::vector<double> ur;  // distinct radii
    uid.assign(n, 0);
    {
        std::map<double, int> seen;
        for (int i = 0; i < n; ++i) {
            auto it = seen.find(c->h_a[i]);
            if (it == seen.end()) {
                it = seen.emplace(c->h_a[i], (int)ur.size()).first;
                ur.push_back(c->h_a[i]);
            }
            uid[i] = it->second;
        }
    }
    const int nu = (int)ur.size();
    const long long cap_nodes = 1LL << 22;  // nodes per pass
    const int G = (int)std::max(1LL, std::min((long long)NM, cap_nodes / ((long long)nu * c->npn)));
    const int ns = nu * G;
    std::vector<double> cc((size_t)ns * 3, 0.0), aa(ns);
    std::vector<int> ps(ns + 1);
    for (int j = 0; j < ns; ++j) {
        aa[j] = ur[j / G];
        ps[j] = j;
    }
    ps[ns] = ns;
    sbie_ctx* sc = nullptr;
    CKS(create_part(o, ns, cc.data(), aa.data(), ps, c->stream, &sc));
    std::vector<double> ZS, ZA;
    lowmode_tables(c->p, ZS, ZA);
    double *dZS = nullptr, *dZA = nullptr, *dB = nullptr;
    sbie_status st = SBIE_OK;
    if (dmalloc(&dZS, ZS.size()) != cudaSuccess || dmalloc(&dZA, ZA.size()) != cudaSuccess ||
        dmalloc(&dB, (size_t)nu * blk) != cudaSuccess)
        st = fail(c, SBIE_ERR_OOM, "own-block probe buffers");
    Lu.assign((size_t)nu * blk, 0.0);
    cudaError_t e = cudaSuccess;
    if (st == SBIE_OK) {
        e = h2d(sc->stream, dZS, ZS.data(), ZS.size());
        if (e == cudaSuccess) e = h2d(sc->stream, dZA, ZA.data(), ZA.size());
        for (int b0 = 0; b0 < NM && e == cudaSuccess && st == SBIE_OK; b0 += G) {
            e = launch_probe_density_multi(sc, G, b0, dZS, sc->d_in);
            if (e == cudaSuccess) {
                st = apply_dev(sc, op, kModeF64, sc->d_in, sc->d_out);
                if (st != SBIE_OK) c->err = sc->err;
            }
            if (st == SBIE_OK && e == cudaSuccess) e = launch_probe_analysis_multi(sc, G, b0, dZA, sc->d_out, dB);
        }
        if (e == cudaSuccess && st == SBIE_OK) e = d2h(sc->stream, Lu.data(), dB, Lu.size());
        if (e != cudaSuccess && st == SBIE_OK) st = fail(c, SBIE_ERR_CUDA, std::string("own blocks: ") + cudaGetErrorString(e));
    }
    for (double* p : {dZS, dZA, dB})
        if (p) cudaFree(p);
    free_all(sc);
    delete sc;
    return st;
}

sbie_status precond_setup(sbie_ctx* c, int op, int kind, const PairNet* net) {
    auto t0 = std::chrono::steady_clock::now();
    PrecState& P = c->prec[prec_slot(op)];
    const int n = c->n, NM = kLowModes;
    const size_t blk = (size_t)NM * NM;
    std::vector<double> ZS, ZA;
    lowmode_tables(c->p, ZS, ZA);
    std::vector<int4> modes = low_mode_table();
    // undirected close pairs (the close-pair relation is symmetric)
    std::vector<std::pair<int, int>> pairs;
    for (int i = 0; i < n; ++i)
        for (int e = c->h_near_ptr[i]; e < c->h_near_ptr[i + 1]; ++e)
            if (c->h_near_idx[e] > i) pairs.push_back({i, c->h_near_idx[e]});
    // the network is used only inside the input range it was trained on; a
    // pair outside it is left out of the pair systems (not extrapolated)
    if (kind == 1) {
        std::vector<std::pair<int, int>> kept;
        for (const auto& pr : pairs) {
            const double* ca = &c->h_c[3 * pr.first];
            const double* cb = &c->h_c[3 * pr.second];
            const float d = (float)std::sqrt((cb[0] - ca[0]) * (cb[0] - ca[0]) + (cb[1] - ca[1]) * (cb[1] - ca[1]) +
                                             (cb[2] - ca[2]) * (cb[2] - ca[2]));
            const float x0[kMlpIn] = {0.f, 0.f, d, (float)c->h_a[pr.first], (float)c->h_a[pr.second]};
            const float x1[kMlpIn] = {0.f, 0.f, d, (float)c->h_a[pr.second], (float)c->h_a[pr.first]};
            if (net->covers(x0) && net->covers(x1)) kept.push_back(pr);
        }
        P.n_dropped = (int)(pairs.size() - kept.size());
        pairs.swap(kept);
    }
    const int np = (int)pairs.size();
    // per-sphere lists of the preconditioner's pairs: partner and pair index
    std::vector<int> pp_ptr(n + 1, 0), pp_idx(std::max(1, 2 * np)), pp_pair(std::max(1, 2 * np));
    for (const auto& pr : pairs) {
        ++pp_ptr[pr.first + 1];
        ++pp_ptr[pr.second + 1];
    }
    for (int i = 0; i < n; ++i) pp_ptr[i + 1] += pp_ptr[i];
    {
        std::vector<int> cur(pp_ptr.begin(), pp_ptr.end() - 1);
        for (int q = 0; q < np; ++q) {
            const int a = pairs[q].first, b = pairs[q].second;
            pp_idx[cur[a]] = b;
            pp_pair[cur[a]++] = q;
            pp_idx[cur[b]] = a;
            pp_pair[cur[b]++] = q;
        }
    }
    // own blocks L_i: single-sphere problems
    sbie_opts o = c->opts;
    o.use_learned_precond = 0;
    o.stream = nullptr;
    std::vector<double> Lu;
    std::vector<int> uid;
    sbie_status st = own_blocks(c, o, op, Lu, uid);
    CKS(st);
    // pair blocks B_ab (target a <- source b) and B_ba
    std::vector<double> Bab, Bba;
    if (kind == 2 && np > 0) {
        Bab.resize((size_t)np * blk);
        Bba.resize((size_t)np * blk);
        std::vector<double> cc((size_t)np * 6), aa((size_t)np * 2);
        std::vector<int> ps(np + 1);
        for (int q = 0; q < np; ++q) {
            for (int d = 0; d < 3; ++d) {
                cc[6 * q + d] = c->h_c[3 * pairs[q].first + d];
                cc[6 * q + 3 + d] = c->h_c[3 * pairs[q].second + d];
            }
            aa[2 * q] = c->h_a[pairs[q].first];
            aa[2 * q + 1] = c->h_a[pairs[q].second];
            ps[q] = 2 * q;
        }
        ps[np] = 2 * np;
        sbie_ctx* pc = nullptr;
        CKS(create_part(o, 2 * np, cc.data(), aa.data(), ps, c->stream, &pc));
        std::vector<double> PB;
        st = probe_blocks(pc, op, 2, 2, PB, kModeF32);  // the pair systems are FP32
        if (st != SBIE_OK) c->err = pc->err;
        const size_t per = (size_t)2 * np * blk;
        if (st == SBIE_OK)
            for (int q = 0; q < np; ++q) {
                std::memcpy(Bba.data() + q * blk, PB.data() + 0 * per + (2 * q + 1) * blk, sizeof(double) * blk);
                std::memcpy(Bab.data() + q * blk, PB.data() + 1 * per + (2 * q + 0) * blk, sizeof(double) * blk);
            }
        free_all(pc);
        delete pc;
        CKS(st);
    }
    // learned blocks: the network's inputs, and per direction the pair frame's
    // low-mode rotation as its degree blocks (R from Q, Ri from Q^T)
    constexpr int kDc = 165;
    std::vector<float> X, Dr, Di;
    if (kind == 1 && np > 0) {
        X.assign((size_t)2 * np * kMlpIn, 0.f);
        Dr.resize((size_t)2 * np * kDc);
        Di.resize((size_t)2 * np * kDc);
        std::vector<double> Qs((size_t)2 * np * 9);
        for (int q = 0; q < np; ++q) {
            const int a = pairs[q].first, b = pairs[q].second;
            double d;
            pair_frame(&c->h_c[3 * a], &c->h_c[3 * b], &Qs[(2 * q) * 9], &d);      // a -> b
            pair_frame(&c->h_c[3 * b], &c->h_c[3 * a], &Qs[(2 * q + 1) * 9], &d);  // b -> a
            float* x0 = &X[(2 * q) * kMlpIn];
            x0[2] = (float)d; x0[3] = (float)c->h_a[a]; x0[4] = (float)c->h_a[b];
            float* x1 = &X[(2 * q + 1) * kMlpIn];
            x1[2] = (float)d; x1[3] = (float)c->h_a[b]; x1[4] = (float)c->h_a[a];
        }
        parallel_for(2 * np, [&](int t0, int t1) {
            for (int t = t0; t < t1; ++t) {
                const double* Q = &Qs[(size_t)t * 9];
                double Qt[9];
                for (int r = 0; r < 3; ++r)
                    for (int s = 0; s < 3; ++s) Qt[3 * r + s] = Q[3 * s + r];
                lowmode_rotation_blocks(Q, &Dr[(size_t)t * kDc]);
                lowmode_rotation_blocks(Qt, &Di[(size_t)t * kDc]);
            }
        });
    }
    bool ok = dmalloc(&P.d_pp_ptr, pp_ptr.size()) == cudaSuccess && dmalloc(&P.d_pp_idx, pp_idx.size()) == cudaSuccess &&
              dmalloc(&P.d_pp_pair, pp_pair.size()) == cudaSuccess &&
              dmalloc(&P.d_pinv, (size_t)std::max(1, np) * 4 * blk) == cudaSuccess &&
              dmalloc(&P.d_sinv, (size_t)n * blk) == cudaSuccess;
    const bool tables = !c->d_ZS;
    if (tables)
        ok = ok && dmalloc(&c->d_ZS, ZS.size()) == cudaSuccess && dmalloc(&c->d_ZA, ZA.size()) == cudaSuccess &&
             dmalloc(&c->d_modes, modes.size()) == cudaSuccess && dmalloc(&c->d_low, (size_t)n * NM) == cudaSuccess &&
             dmalloc(&c->d_lowe, (size_t)n * NM) == cudaSuccess;
    if (!ok) return fail(c, SBIE_ERR_OOM, "preconditioner buffers");
    int* d_bad = nullptr;
    CK(cudaMalloc(&d_bad, sizeof(int)));
    CK(cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream));
    if (tables) {
        CK(h2d(c->stream, c->d_ZS, ZS.data(), ZS.size()));
        if (c->opts.prec == SBIE_MIXED) {  // FP32 copy for the FP32 inner solves
            std::vector<float> ZSf(ZS.begin(), ZS.end());
            if (dmalloc(&c->d_ZSf, ZSf.size()) != cudaSuccess) return fail(c, SBIE_ERR_OOM, "preconditioner buffers");
            CK(h2d(c->stream, c->d_ZSf, ZSf.data(), ZSf.size()));
            CK(cudaStreamSynchronize(c->stream));
        }
        CK(h2d(c->stream, c->d_ZA, ZA.data(), ZA.size()));
        CK(h2d(c->stream, c->d_modes, modes.data(), modes.size()));
    }
    CK(h2d(c->stream, P.d_pp_ptr, pp_ptr.data(), pp_ptr.size()));
    CK(h2d(c->stream, P.d_pp_idx, pp_idx.data(), pp_idx.size()));
    CK(h2d(c->stream, P.d_pp_pair, pp_pair.data(), pp_pair.size()));
    if (kind == 1) {
        // pair systems and own systems assembled on the device from the
        // network's outputs, which never leave it
        std::vector<float> Luf(Lu.begin(), Lu.end());
        std::vector<int2> pr2((size_t)std::max(1, np));
        for (int q = 0; q < np; ++q) pr2[q] = make_int2(pairs[q].first, pairs[q].second);
        float *dLu = nullptr, *dY = nullptr, *dDr = nullptr, *dDi = nullptr, *dmean = nullptr, *dsd = nullptr;
        int* duid = nullptr;
        int2* dpr = nullptr;
        cudaError_t e = cudaSuccess;
        if (dmalloc(&dLu, Luf.size()) != cudaSuccess || dmalloc(&duid, uid.size()) != cudaSuccess) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = h2d(c->stream, dLu, Luf.data(), Luf.size());
        if (e == cudaSuccess) e = h2d(c->stream, duid, uid.data(), uid.size());
        if (e == cudaSuccess && np > 0) {
            if (dmalloc(&dY, (size_t)2 * np * blk) != cudaSuccess || dmalloc(&dDr, Dr.size()) != cudaSuccess ||
                dmalloc(&dDi, Di.size()) != cudaSuccess || dmalloc(&dmean, blk) != cudaSuccess ||
                dmalloc(&dsd, blk) != cudaSuccess || dmalloc(&dpr, pr2.size()) != cudaSuccess)
                e = cudaErrorMemoryAllocation;
            if (e == cudaSuccess) e = h2d(c->stream, dDr, Dr.data(), Dr.size());
            if (e == cudaSuccess) e = h2d(c->stream, dDi, Di.data(), Di.size());
            if (e == cudaSuccess) e = h2d(c->stream, dmean, net->out_mean.data(), blk);
            if (e == cudaSuccess) e = h2d(c->stream, dsd, net->out_std.data(), blk);
            if (e == cudaSuccess) e = h2d(c->stream, dpr, pr2.data(), pr2.size());
            if (e == cudaSuccess) {
                const sbie_status sn = net_forward_dev(*net, X, c->stream, dY);
                if (sn != SBIE_OK) e = cudaErrorUnknown;
            }
            if (e == cudaSuccess)
                e = launch_pair_systems(c->stream, np, dpr, duid, dLu, dY, dmean, dsd, dDr, dDi, P.d_pinv);
        }
        if (e == cudaSuccess) e = launch_own_systems(c->stream, n, duid, dLu, P.d_sinv);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        for (void* p : {(void*)dLu, (void*)dY, (void*)dDr, (void*)dDi, (void*)dmean, (void*)dsd, (void*)duid, (void*)dpr})
            if (p) cudaFree(p);
        if (e != cudaSuccess) {
            cudaFree(d_bad);
            return fail(c, SBIE_ERR_CUDA, std::string("learned pair systems: ") + cudaGetErrorString(e));
        }
    } else {
        // exact blocks: pair systems [[L_a, B_ab], [B_ba, L_b]] and own blocks assembled here
        std::vector<float> A((size_t)std::max(1, np) * 4 * blk), S((size_t)n * blk);
        parallel_for(np, [&](int q0, int q1) {
            for (int q = q0; q < q1; ++q) {
                const double* La = &Lu[(size_t)uid[pairs[q].first] * blk];
                const double* Lb = &Lu[(size_t)uid[pairs[q].second] * blk];
                float* M = A.data() + q * 4 * blk;
                for (int r = 0; r < NM; ++r)
                    for (int s = 0; s < NM; ++s) {
                        M[r * 2 * NM + s] = (float)La[r * NM + s];
                        M[r * 2 * NM + NM + s] = (float)Bab[q * blk + r * NM + s];
                        M[(NM + r) * 2 * NM + s] = (float)Bba[q * blk + r * NM + s];
                        M[(NM + r) * 2 * NM + NM + s] = (float)Lb[r * NM + s];
                    }
            }
        });
        for (int i = 0; i < n; ++i)
            for (size_t e = 0; e < blk; ++e) S[(size_t)i * blk + e] = (float)Lu[(size_t)uid[i] * blk + e];
        CK(h2d(c->stream, P.d_pinv, A.data(), A.size()));
        CK(h2d(c->stream, P.d_sinv, S.data(), S.size()));
    }
    CK(launch_gauss_jordan(c->stream, 2 * NM, np, P.d_pinv, d_bad));
    CK(launch_gauss_jordan(c->stream, NM, n, P.d_sinv, d_bad));
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(d_bad);
    if (bad) return fail(c, SBIE_ERR_NUMERIC, "singular pair system in the preconditioner");
    if (c->opts.prec == SBIE_MIXED) {
        // H and the low-mode analysis of the FP32 inner solves as one GEMM
        const cudaError_t e = self_gemm_build(c, kSelfPrec);
        if (e != cudaSuccess)
            return fail(c, SBIE_ERR_CUDA, std::string("preconditioner matrix: ") + cudaGetErrorString(e));
        // the FP32 coarse correction's entry owners and per-entry products
        P.n_entries = pp_ptr[n];
        std::vector<int> own(std::max(1, P.n_entries));
        for (int i = 0; i < n; ++i)
            for (int ee = pp_ptr[i]; ee < pp_ptr[i + 1]; ++ee) own[ee] = i;
        if (dmalloc(&P.d_pp_own, own.size()) != cudaSuccess ||
            dmalloc(&P.d_cpart, (size_t)std::max(1, P.n_entries) * kLowModes) != cudaSuccess)
            return fail(c, SBIE_ERR_OOM, "coarse-correction buffers");
        CK(h2d(c->stream, P.d_pp_own, own.data(), own.size()));
        CK(cudaStreamSynchronize(c->stream));
    }
    P.n_pairs = np;
    P.kind = kind;
    P.built = true;
    P.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ++g_graph_epoch;  // cycle graphs capture the preconditioner's buffers
    return SBIE_OK;
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
    o->use_graphs = 1;
    return SBIE_OK;
}

sbie_status sphere_bie_create(int n, const double* centres, const double* radii, const sbie_opts* opts,
                              sbie_ctx** out) {
    int one = n;
    return sphere_bie_create_batch(1, &one, opts ? &opts->p : nullptr, centres, radii, opts, out);
}

sbie_status sphere_bie_create_batch(int n_problems, const int* n_spheres, const int* p_per_problem,
                                    const double* centres, const double* radii, const sbie_opts* opts, sbie_ctx** out) {
    if (!out) return fail(nullptr, SBIE_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_problems < 1 || !n_spheres || !p_per_problem || !centres || !radii || !opts)
        return fail(nullptr, SBIE_ERR_ARG, "need n_problems >= 1 and non-NULL arrays");
    CKS(check_opts(opts));
    const auto t_create0 = std::chrono::steady_clock::now();
    auto create_ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_create0).count();
    };
    long long ntot = 0;
    for (int q = 0; q < n_problems; ++q) {
        if (n_spheres[q] < 1) return fail(nullptr, SBIE_ERR_ARG, "every problem needs n >= 1 spheres");
        if (p_per_problem[q] < 1 || p_per_problem[q] > kMaxP) return fail(nullptr, SBIE_ERR_ARG, "p must be in [1, 24]");
        if (opts->use_learned_precond > 0 && p_per_problem[q] < kPrecL)
            return fail(nullptr, SBIE_ERR_ARG, "the pair preconditioner needs p >= 4");
        ntot += n_spheres[q];
    }
    if (ntot > (1LL << 30)) return fail(nullptr, SBIE_ERR_ARG, "too many spheres");
    if (!finite_all(centres, (size_t)ntot * 3) || !finite_all(radii, ntot))
        return fail(nullptr, SBIE_ERR_ARG, "non-finite centre or radius");
    for (long long i = 0; i < ntot; ++i)
        if (!(radii[i] > 0.0)) return fail(nullptr, SBIE_ERR_ARG, "radii must be positive");
    std::vector<long long> usph(n_problems + 1, 0), unode(n_problems + 1, 0);
    for (int q = 0; q < n_problems; ++q) {
        usph[q + 1] = usph[q] + n_spheres[q];
        unode[q + 1] = unode[q] + (long long)n_spheres[q] * (p_per_problem[q] + 1) * (2 * p_per_problem[q] + 2);
    }
    // overlap check for every problem before any device work
    for (int q = 0; q < n_problems; ++q)
        for (long long i = usph[q]; i < usph[q + 1]; ++i)
            for (long long k = i + 1; k < usph[q + 1]; ++k) {
                double dx = centres[3 * i] - centres[3 * k], dy = centres[3 * i + 1] - centres[3 * k + 1],
                       dz = centres[3 * i + 2] - centres[3 * k + 2];
                if (std::sqrt(dx * dx + dy * dy + dz * dz) - radii[i] - radii[k] <= 0.0)
                    return fail(nullptr, SBIE_ERR_OVERLAP,
                                "problem " + std::to_string(q) + ": spheres " + std::to_string(i - usph[q]) + " and " +
                                    std::to_string(k - usph[q]) + " overlap or touch");
            }
    // the pair networks are read (and checked) here; the preconditioner of an
    // operator is built at the first solve with it
    std::shared_ptr<PairNetSet> nets;
    if (opts->use_learned_precond == 1) {
        nets = std::make_shared<PairNetSet>();
        CKS(net_load(opts->mlp_weights_path, *nets));
    }
    // group problems by VSH order
    std::vector<int> orders(p_per_problem, p_per_problem + n_problems);
    std::sort(orders.begin(), orders.end());
    orders.erase(std::unique(orders.begin(), orders.end()), orders.end());
    if (orders.size() == 1) {
        std::vector<int> prob_sph(n_problems + 1);
        for (int q = 0; q <= n_problems; ++q) prob_sph[q] = (int)usph[q];
        sbie_opts o = *opts;
        o.p = orders[0];
        sbie_ctx* c = nullptr;
        CKS(create_part(o, (int)ntot, centres, radii, prob_sph, nullptr, &c));
        c->nets = nets;
        c->t_create_ms = create_ms();
        *out = c;
        return SBIE_OK;
    }
    sbie_ctx* top = new (std::nothrow) sbie_ctx();
    if (!top) return fail(nullptr, SBIE_ERR_OOM, "host allocation");
    top->opts = *opts;
    top->is_batch = true;
    auto bail = [&](sbie_status s, const std::string& m) {
        g_last_error = m;
        free_all(top);
        delete top;
        return s;
    };
    cudaError_t e = cudaGetDevice(&top->device);
    if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (opts->stream) {
        top->stream = (cudaStream_t)opts->stream;
    } else {
        e = cudaStreamCreateWithFlags(&top->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        top->own_stream = true;
    }
    top->prob_part.assign(n_problems, 0);
    top->prob_local.assign(n_problems, 0);
    top->prob_user_node = unode;
    top->prob_user_sph = usph;
    long long off3 = 0;
    std::vector<int> node_prob;
    top->seg3.assign(1, 0);
    int pbase = 0;
    for (size_t s = 0; s < orders.size(); ++s) {
        std::vector<double> cc, aa;
        std::vector<int> prob_sph(1, 0);
        int local = 0;
        for (int q = 0; q < n_problems; ++q) {
            if (p_per_problem[q] != orders[s]) continue;
            cc.insert(cc.end(), centres + 3 * usph[q], centres + 3 * usph[q + 1]);
            aa.insert(aa.end(), radii + usph[q], radii + usph[q + 1]);
            prob_sph.push_back(prob_sph.back() + n_spheres[q]);
            top->prob_part[q] = (int)s;
            top->prob_local[q] = local++;
        }
        sbie_opts o = *opts;
        o.p = orders[s];
        o.stream = top->stream;
        sbie_ctx* part = nullptr;
        sbie_status st = create_part(o, (int)aa.size(), cc.data(), aa.data(), prob_sph, top->stream, &part);
        if (st != SBIE_OK) return bail(st, g_last_error);
        top->parts.push_back(part);
        top->part_off3.push_back(off3);
        for (size_t k = 1; k < part->seg3.size(); ++k) top->seg3.push_back(off3 + part->seg3[k]);
        for (int k = 0; k < part->n_prob; ++k)
            node_prob.insert(node_prob.end(), (size_t)(part->h_prob_sph[k + 1] - part->h_prob_sph[k]) * part->npn,
                             pbase + k);
        pbase += part->n_prob;
        off3 += part->N * 3;
        top->n += part->n;
        top->n_near += part->n_near;
    }
    top->N = off3 / 3;
    top->n_prob = n_problems;
    top->sm_count = top->parts[0]->sm_count;
    const long long N = top->N;
    bool ok = true;
    for (double** p : {&top->d_in, &top->d_out, &top->d_tmp, &top->d_tmp2, &top->d_xsol, &top->d_rhs, &top->d_res})
        ok &= dmalloc(p, 3 * (size_t)N) == cudaSuccess;
    ok &= dmalloc(&top->d_small, 3 * (size_t)top->n * 6 + 32) == cudaSuccess;
    ok &= dmalloc(&top->d_node_prob, (size_t)N) == cudaSuccess;
    ok &= dmalloc(&top->d_seg3, top->seg3.size()) == cudaSuccess;
    if (!ok) return bail(SBIE_ERR_OOM, "device allocation failed");
    e = h2d(top->stream, top->d_node_prob, node_prob.data(), (size_t)N);
    if (e == cudaSuccess)
        e = h2d(top->stream, top->d_seg3, top->seg3.data(), top->seg3.size());
    if (e != cudaSuccess) return bail(SBIE_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e));
    top->nets = nets;
    top->err = "no error";
    top->t_create_ms = create_ms();
    *out = top;
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
    Sys S = sys_of(c);
    std::vector<double> x4, n4, ix((size_t)c->N * 3), inr((size_t)c->N * 3), iw((size_t)c->N);
    for (size_t s = 0; s < S.parts.size(); ++s) {
        sbie_ctx* q = S.parts[s];
        x4.resize(4 * (size_t)q->N);
        n4.resize(4 * (size_t)q->N);
        CK(d2h(q->stream, x4.data(), q->d_x, x4.size()));
        CK(d2h(q->stream, n4.data(), q->d_nrm64, n4.size()));
        const long long o = S.off3[s] / 3;
        for (long long i = 0; i < q->N; ++i) {
            for (int d = 0; d < 3; ++d) {
                ix[3 * (o + i) + d] = x4[4 * i + d];
                inr[3 * (o + i) + d] = n4[4 * i + d];
            }
            iw[o + i] = x4[4 * i + 3];
        }
    }
    // internal -> user order (identity unless the batch holds several VSH orders)
    auto put = [&](double* dst, const std::vector<double>& src, int width) {
        if (!dst) return;
        if (!c->is_batch) {
            std::memcpy(dst, src.data(), sizeof(double) * src.size());
            return;
        }
        for (int q = 0; q < c->n_prob; ++q) {
            sbie_ctx* part = c->parts[c->prob_part[q]];
            long long inode = c->part_off3[c->prob_part[q]] / 3 +
                              (long long)part->h_prob_sph[c->prob_local[q]] * part->npn;
            long long cnt = c->prob_user_node[q + 1] - c->prob_user_node[q];
            std::memcpy(dst + width * c->prob_user_node[q], src.data() + width * inode, sizeof(double) * width * cnt);
        }
    };
    put(xyz, ix, 3);
    put(normals, inr, 3);
    put(weights, iw, 1);
    return SBIE_OK;
}

sbie_status sphere_bie_apply_operator(sbie_ctx* c, sbie_op op, const double* density, double* out) {
    if (!c) return SBIE_ERR_ARG;
    if (!density || !out) return fail(c, SBIE_ERR_ARG, "NULL density or out");
    if (op < SBIE_OP_S || op > SBIE_OP_SQUIRMER) return fail(c, SBIE_ERR_ARG, "bad operator");
    if (density == out) return fail(c, SBIE_ERR_ARG, "density and out must not alias");
    const int mode = c->opts.prec == SBIE_MIXED ? kModeF32 : hi_mode(c);
    Sys S = sys_of(c);
    CKS(ensure_self_gemm(S));
    if (op == SBIE_OP_SQUIRMER) CKS(ensure_squirmer_buffers(S));
    const bool direct = c->opts.mem_kind == 1 && !c->is_batch;
    if (direct) {
        CKS(apply_sys(S, op, mode, density, out));
    } else {
        CKS(to_internal(c, density, c->d_in, true));
        CKS(apply_sys(S, op, mode, c->d_in, c->d_out));
        CKS(to_user(c, c->d_out, out, true));
    }
    CK(cudaStreamSynchronize(c->stream));
    return check_self_gemm(S);
}

// Eq. 5.8 for the incident force density rho (device, internal order, [N][3];
// rho must not be c->d_rhs, d_xsol, d_out or d_tmp2): solve
// (1/2 I + K + L) mu = -(1/2 I + K) rho, u = S[mu + rho], rigid projection into
// dv, dw ([n][3] device, internal order).
sbie_status mobility_from_density(const Sys& S, const double* rho, double* dv, double* dw, sbie_solve_info* inf) {
    sbie_ctx* c = S.top;
    const long long n3 = S.n3;
    double* b = c->d_rhs;
    double* mu = c->d_xsol;
    // b = -(1/2 I + K) rho
    CKS(apply_sys(S, SBIE_OP_K, hi_mode(c), rho, b));
    CK(blas_lincomb(c, -0.5, rho, -1.0, b, b, n3));
    sbie_status st = solve_sys(S, SBIE_OP_MOBILITY, b, mu, inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    // u = S[mu + rho] on every sphere; rigid projection
    CK(blas_lincomb(c, 1.0, mu, 1.0, rho, c->d_tmp2, n3));
    CKS(apply_sys(S, SBIE_OP_S, hi_mode(c), c->d_tmp2, c->d_out));
    long long sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        CK(launch_rigid_projection(S.parts[s], c->d_out + S.off3[s], dv + 3 * sph_off, dw + 3 * sph_off));
        sph_off += S.parts[s]->n;
    }
    return st;
}

sbie_status sphere_bie_solve_mobility(sbie_ctx* c, const double* forces, const double* torques, double* vel,
                                      double* omega, sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!forces || !torques || !vel || !omega) return fail(c, SBIE_ERR_ARG, "NULL argument");
    auto t0 = std::chrono::steady_clock::now();
    Sys S = sys_of(c);
    const long long launches0 = total_launches(S);
    const long long n3 = S.n3;
    double* dF = c->d_small;
    double* dT = dF + 3 * c->n;
    double* dv = dT + 3 * c->n;
    double* dw = dv + 3 * c->n;
    CKS(to_internal(c, forces, dF, false));
    CKS(to_internal(c, torques, dT, false));
    double* rho = c->d_in;
    long long sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        CK(launch_rho(S.parts[s], dF + 3 * sph_off, dT + 3 * sph_off, rho + S.off3[s]));
        sph_off += S.parts[s]->n;
    }
    sbie_solve_info inf{};
    sbie_status st = mobility_from_density(S, rho, dv, dw, &inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    CKS(to_user(c, dv, vel, false));
    CKS(to_user(c, dw, omega, false));
    CK(cudaStreamSynchronize(c->stream));
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    inf.t_setup_ms = c->t_create_ms;
    c->has_solution = true;
    inf.kernel_launches = total_launches(S) - launches0;
    if (info) *info = inf;
    return st;
}

sbie_status sphere_bie_solve_resistance(sbie_ctx* c, const double* vel, const double* omega, const double* bg_u0,
                                        const double* bg_grad, double* forces, double* torques, sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!vel || !omega || !forces || !torques) return fail(c, SBIE_ERR_ARG, "NULL argument");
    if (bg_u0 && !finite_all(bg_u0, 3)) return fail(c, SBIE_ERR_ARG, "non-finite u0");
    if (bg_grad && !finite_all(bg_grad, 9)) return fail(c, SBIE_ERR_ARG, "non-finite velocity gradient");
    auto t0 = std::chrono::steady_clock::now();
    Sys S = sys_of(c);
    const long long launches0 = total_launches(S);
    double* dv = c->d_small;
    double* dw = dv + 3 * c->n;
    double* dF = dw + 3 * c->n;
    double* dT = dF + 3 * c->n;
    CKS(to_internal(c, vel, dv, false));
    CKS(to_internal(c, omega, dw, false));
    double* b = c->d_rhs;
    double* psi = c->d_xsol;
    long long sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        CK(launch_resistance_rhs(S.parts[s], dv + 3 * sph_off, dw + 3 * sph_off, bg_u0, bg_grad, b + S.off3[s]));
        sph_off += S.parts[s]->n;
    }
    sbie_solve_info inf{};
    sbie_status st = solve_sys(S, SBIE_OP_RESISTANCE, b, psi, &inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        sbie_ctx* q = S.parts[s];
        CK(launch_moments(q, psi + S.off3[s]));
        // forces / torques from the moments [n][6]
        CK(cudaMemcpy2DAsync(dF + 3 * sph_off, sizeof(double) * 3, q->d_mom, sizeof(double) * 6, sizeof(double) * 3,
                             q->n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpy2DAsync(dT + 3 * sph_off, sizeof(double) * 3, q->d_mom + 3, sizeof(double) * 6, sizeof(double) * 3,
                             q->n, cudaMemcpyDeviceToDevice, c->stream));
        sph_off += q->n;
    }
    CKS(to_user(c, dF, forces, false));
    CKS(to_user(c, dT, torques, false));
    CK(cudaStreamSynchronize(c->stream));
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    inf.t_setup_ms = c->t_create_ms;
    c->has_solution = true;
    inf.kernel_launches = total_launches(S) - launches0;
    if (info) *info = inf;
    return st;
}

sbie_status sphere_bie_solve_porous(sbie_ctx* c, const double* bg_u0, const double* bg_grad, double* forces,
                                    double* torques, sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!forces || !torques) return fail(c, SBIE_ERR_ARG, "NULL argument");
    if (bg_u0 && !finite_all(bg_u0, 3)) return fail(c, SBIE_ERR_ARG, "non-finite u0");
    if (bg_grad && !finite_all(bg_grad, 9)) return fail(c, SBIE_ERR_ARG, "non-finite velocity gradient");
    auto t0 = std::chrono::steady_clock::now();
    Sys S = sys_of(c);
    const long long launches0 = total_launches(S);
    double* dF = c->d_small;
    double* dT = dF + 3 * c->n;
    double* dz = dT + 3 * c->n;  // zero rigid motions: b = -u_inf
    CK(cudaMemsetAsync(dz, 0, sizeof(double) * 3 * c->n, c->stream));
    double* b = c->d_rhs;
    double* mu = c->d_xsol;
    long long sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        CK(launch_resistance_rhs(S.parts[s], dz + 3 * sph_off, dz + 3 * sph_off, bg_u0, bg_grad, b + S.off3[s]));
        sph_off += S.parts[s]->n;
    }
    sbie_solve_info inf{};
    sbie_status st = solve_sys(S, SBIE_OP_POROUS, b, mu, &inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        sbie_ctx* q = S.parts[s];
        CK(launch_moments(q, mu + S.off3[s]));
        CK(cudaMemcpy2DAsync(dF + 3 * sph_off, sizeof(double) * 3, q->d_mom, sizeof(double) * 6, sizeof(double) * 3,
                             q->n, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpy2DAsync(dT + 3 * sph_off, sizeof(double) * 3, q->d_mom + 3, sizeof(double) * 6, sizeof(double) * 3,
                             q->n, cudaMemcpyDeviceToDevice, c->stream));
        sph_off += q->n;
    }
    CKS(to_user(c, dF, forces, false));
    CKS(to_user(c, dT, torques, false));
    CK(cudaStreamSynchronize(c->stream));
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    inf.t_setup_ms = c->t_create_ms;
    c->has_solution = true;
    inf.kernel_launches = total_launches(S) - launches0;
    if (info) *info = inf;
    return st;
}

sbie_status sphere_bie_solve_squirmer(sbie_ctx* c, const double* slip, double* vel, double* omega,
                                      sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!slip || !vel || !omega) return fail(c, SBIE_ERR_ARG, "NULL argument");
    auto t0 = std::chrono::steady_clock::now();
    Sys S = sys_of(c);
    const long long launches0 = total_launches(S);
    CKS(ensure_squirmer_buffers(S));
    double* dv = c->d_small;
    double* dw = dv + 3 * c->n;
    double* b = c->d_rhs;
    double* mu = c->d_xsol;
    CKS(to_internal(c, slip, b, true));
    sbie_solve_info inf{};
    sbie_status st = solve_sys(S, SBIE_OP_SQUIRMER, b, mu, &inf);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    // rigid velocities from the rigid part of mu; keep mu - P mu as the density
    long long sph_off = 0;
    for (size_t s = 0; s < S.parts.size(); ++s) {
        sbie_ctx* q = S.parts[s];
        CK(launch_rigid_projection(q, mu + S.off3[s], dv + 3 * sph_off, dw + 3 * sph_off));
        CK(launch_moments(q, mu + S.off3[s]));
        CK(launch_rigid_split(q, mu + S.off3[s], q->d_sq, q->d_sq + 3 * q->N));
        CK(cudaMemcpyAsync(mu + S.off3[s], q->d_sq, sizeof(double) * 3 * q->N, cudaMemcpyDeviceToDevice, c->stream));
        sph_off += q->n;
    }
    CKS(to_user(c, dv, vel, false));
    CKS(to_user(c, dw, omega, false));
    CK(cudaStreamSynchronize(c->stream));
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    inf.t_setup_ms = c->t_create_ms;
    c->has_solution = true;
    inf.kernel_launches = total_launches(S) - launches0;
    if (info) *info = inf;
    return st;
}

namespace {

__global__ void scalar_to_vec_kernel(long long N, const double* __restrict__ q, double* __restrict__ v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    v[3 * i] = q[i];
    v[3 * i + 1] = 0.0;
    v[3 * i + 2] = 0.0;
}

__global__ void vec_to_scalar_kernel(long long N, const double* __restrict__ v, double* __restrict__ q) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) q[i] = v[3 * i];
}

sbie_status ensure_laplace_buffers(sbie_ctx* c) {
    const int P1 = c->p + 1;
    if (!c->d_lcoef && dmalloc(&c->d_lcoef, (size_t)c->n * P1 * P1 * 2) != cudaSuccess)
        return fail(c, SBIE_ERR_OOM, "Laplace coefficient buffer");
    if (!c->d_sq && dmalloc(&c->d_sq, 6 * (size_t)c->N) != cudaSuccess)
        return fail(c, SBIE_ERR_OOM, "Laplace work vectors");
    return SBIE_OK;
}

}  // namespace

sbie_status sphere_bie_apply_laplace(sbie_ctx* c, int op, const double* q, double* out) {
    if (!c) return SBIE_ERR_ARG;
    if (!q || !out || q == out) return fail(c, SBIE_ERR_ARG, "NULL or aliased density / out");
    if (op < kLapSL || op > kLapKL) return fail(c, SBIE_ERR_ARG, "op must be 0 (S^L), 1 (D^L) or 2 (K^L)");
    if (c->is_batch) return fail(c, SBIE_ERR_ARG, "Laplace operators take a single-order context");
    CKS(ensure_laplace_buffers(c));
    const long long N = c->N;
    const unsigned nb = (unsigned)((N + 255) / 256);
    double* qv = c->d_sq;  // [N][3] with the density in component 0
    const double* qs = q;
    if (c->opts.mem_kind == 0) {
        CK(h2d(c->stream, c->d_tmp2, q, (size_t)N));
        qs = c->d_tmp2;
    }
    scalar_to_vec_kernel<<<nb, 256, 0, c->stream>>>(N, qs, qv); ++c->n_launch;
    CK(cudaGetLastError());
    CK(laplace_apply(c, op, qv, c->d_out));
    double* os = c->opts.mem_kind == 0 ? c->d_tmp2 : out;
    vec_to_scalar_kernel<<<nb, 256, 0, c->stream>>>(N, c->d_out, os); ++c->n_launch;
    CK(cudaGetLastError());
    if (c->opts.mem_kind == 0) CK(d2h(c->stream, out, c->d_tmp2, (size_t)N));
    CK(cudaStreamSynchronize(c->stream));
    return SBIE_OK;
}

sbie_status sphere_bie_solve_mhd(sbie_ctx* c, const double* H0, double eta, double* forces, double* torques,
                                 double* vel, double* omega, sbie_solve_info* info) {
    if (!c) return SBIE_ERR_ARG;
    if (!H0 || !forces || !torques || !vel || !omega) return fail(c, SBIE_ERR_ARG, "NULL argument");
    if (!finite_all(H0, 3) || !std::isfinite(eta) || !(eta > -1.0 && eta < 1.0))
        return fail(c, SBIE_ERR_ARG, "H0 must be finite and -1 < eta < 1");
    if (c->is_batch) return fail(c, SBIE_ERR_ARG, "the magnetostatic problem takes a single-order context");
    auto t0 = std::chrono::steady_clock::now();
    Sys S = sys_of(c);
    const long long launches0 = total_launches(S);
    CKS(ensure_laplace_buffers(c));
    double* q = c->d_sq;                   // magnetic density (component 0)
    double* rho = c->d_sq + 3 * c->N;      // Maxwell traction
    double* dF = c->d_small;
    double* dT = dF + 3 * c->n;
    double* dv = dT + 3 * c->n;
    double* dw = dv + 3 * c->n;
    // Eq. 5.13: (1/2 I + eta K^L) q = eta H0 . n
    c->mag_eta = eta;
    CK(launch_magnetic_rhs(c, eta, H0, c->d_rhs));
    sbie_solve_info im{};
    sbie_status st = solve_sys(S, kOpMagnetic, c->d_rhs, c->d_xsol, &im);
    if (st != SBIE_OK && st != SBIE_ERR_NOT_CONVERGED) return st;
    CK(cudaMemcpyAsync(q, c->d_xsol, sizeof(double) * 3 * c->N, cudaMemcpyDeviceToDevice, c->stream));
    // H = H0 - grad S^L[q] outside; traction (H.n) H - |H|^2 n / 2
    CK(laplace_apply(c, kLapGrad, q, rho));
    CK(launch_maxwell_traction(c, H0, rho));
    CK(launch_moments(c, rho));
    CK(cudaMemcpy2DAsync(dF, sizeof(double) * 3, c->d_mom, sizeof(double) * 6, sizeof(double) * 3, c->n,
                         cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpy2DAsync(dT, sizeof(double) * 3, c->d_mom + 3, sizeof(double) * 6, sizeof(double) * 3, c->n,
                         cudaMemcpyDeviceToDevice, c->stream));
    // the traction as the incident force density of the mobility problem (Eq. 5.8)
    sbie_solve_info inf{};
    sbie_status st2 = mobility_from_density(S, rho, dv, dw, &inf);
    if (st2 != SBIE_OK && st2 != SBIE_ERR_NOT_CONVERGED) return st2;
    CKS(to_user(c, dF, forces, false));
    CKS(to_user(c, dT, torques, false));
    CKS(to_user(c, dv, vel, false));
    CKS(to_user(c, dw, omega, false));
    CK(cudaStreamSynchronize(c->stream));
    inf.iters += im.iters;
    inf.restarts += im.restarts;
    inf.graph_cycles += im.graph_cycles;
    inf.rel_residual_true = std::max(inf.rel_residual_true, im.rel_residual_true);
    inf.t_solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    inf.t_setup_ms = c->t_create_ms;
    c->has_solution = true;
    inf.kernel_launches = total_launches(S) - launches0;
    if (info) *info = inf;
    return st != SBIE_OK ? st : st2;
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
    // splits keep the partial sums ([split][N][3] doubles) near 100 MB at most
    const long long max_sp = std::max<long long>(16, std::min<long long>(64, (1LL << 22) / std::max<long long>(1, c->N)));
    const int tpts32[3] = {2, 4, 6}, tpts1[1] = {1};
    const int* tpts = f32 ? tpts32 : tpts1;
    const int ntpt = f32 ? 3 : 1;
    const int ths32[5] = {64, 96, 128, 192, 256}, thsdf[3] = {64, 128, 256};
    const int* ths = f32 ? ths32 : thsdf;
    const int nth = f32 ? 5 : 3;
    const int splits32[8] = {1, 2, 3, 4, 6, 8, 12, 16}, splitsdf[4] = {1, 2, 4, 8};
    const int* splits = f32 ? splits32 : splitsdf;
    const int nsp = f32 ? 8 : 4;
    // short tiles only help small contexts (more source splits)
    const bool small = c->N < 65536;
    const int tiles32[4] = {128, 256, 32, 64}, tilesdf[3] = {128, 32, 64};
    const int* tiles = f32 ? tiles32 : tilesdf;
    const int nti = f32 ? (small ? 4 : 2) : (small ? 3 : 1);
    for (int a = 0; a < ntpt; ++a)
        for (int b = 0; b < nth; ++b) {
            const int tpt = tpts[a], th = ths[b];
            int slots = th * tpt;
            int chunks = (c->npn + slots - 1) / slots;
            double waste = (double)(chunks * slots - c->npn) / c->npn;
            if (waste > 0.30) continue;
            for (int t = 0; t < nti; ++t) {
                // the fixed splits, and those whose grid fills whole waves of
                // resident CTAs (equal-work CTAs: a partial last wave idles SMs)
              int mbs[4] = {0, 0, 0, 0};
              const int nmb = (f32 && th == 64) ? far_f32_builds(tpt, mbs) : 1;
              for (int m = 0; m < nmb; ++m) {
                const int mb = mbs[m];
                std::vector<int> sps(splits, splits + nsp);
                const int occ = far_occupancy(c, k, mode, FarTune{th, tpt, 1, tiles[t], mb});
                if (occ > 0) {
                    const long long wave = (long long)occ * c->sm_count, base = (long long)c->n * chunks;
                    for (int w = 1; w <= 8; ++w) {
                        const long long sp = (w * wave) / base;
                        if (sp >= 1 && sp <= max_sp) sps.push_back((int)sp);
                    }
                }
                std::sort(sps.begin(), sps.end());
                sps.erase(std::unique(sps.begin(), sps.end()), sps.end());
                for (size_t s = 0; s < sps.size(); ++s) {
                    const int sp = sps[s];
                    long long ctas = (long long)c->n * chunks * sp;
                    if (ctas < c->sm_count && s != 0) continue;
                    if (ctas > 64LL * c->sm_count) continue;
                    if ((c->N + sp - 1) / sp < tiles[t]) continue;
                    cands.push_back(Cand{FarTune{th, tpt, sp, tiles[t], mb}, 0.f});
                }
              }
            }
        }
    FarTune* slot = f32 ? &c->tune32[(int)k] : &c->tunedf[(int)k];
    if (cands.empty()) cands.push_back(Cand{*slot, 0.f});
    // the partial-sum buffer must hold the largest split timed, plus the
    // slot the timed reduction writes
    int msp = 1;
    for (const Cand& cd : cands) msp = std::max(msp, cd.t.split);
    CKS(ensure_part(c, msp + 1));
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
    ++g_graph_epoch;
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
        chosen->min_blocks = cands[0].t.minb;
    }
    return SBIE_OK;
}

}  // namespace

extern "C" {

sbie_status sphere_bie_autotune(sbie_ctx* c, sbie_op op, sbie_far_tuning* chosen) {
    if (!c) return SBIE_ERR_ARG;
    if (op < SBIE_OP_S || op > SBIE_OP_SQUIRMER) return fail(c, SBIE_ERR_ARG, "bad operator");
    if (op == SBIE_OP_POROUS || op == SBIE_OP_SQUIRMER) {
        // both layers' far fields; `chosen` reports the double layer's
        CKS(sphere_bie_autotune(c, SBIE_OP_S, nullptr));
        return sphere_bie_autotune(c, SBIE_OP_D, chosen);
    }
    const Kern k = kern_of(op);
    if (chosen) std::memset(chosen, 0, 2 * sizeof(*chosen));
    Sys S = sys_of(c);
    for (sbie_ctx* q : S.parts) {
        sbie_status st = SBIE_OK;
        {
            sbie_ctx* cc = q;
            std::swap(c, cc);
            CKS(ensure_part(c, 16));
            CK(cudaMemsetAsync(c->d_srcf, 0, sizeof(float4) * c->N, c->stream));
            CK(cudaMemsetAsync(c->d_src64, 0, sizeof(double4) * c->N, c->stream));
            if (c->opts.prec == SBIE_MIXED) st = tune_one(c, k, kModeF32, chosen);
            if (st == SBIE_OK && c->opts.prec != SBIE_FP64) st = tune_one(c, k, kModeDF, chosen ? chosen + 1 : nullptr);
            std::swap(c, cc);
        }
        if (st != SBIE_OK) {
            if (q != c) c->err = q->err;
            return st;
        }
    }
    return SBIE_OK;
}

sbie_status sphere_bie_profile(sbie_ctx* c, int enable) {
    if (!c) return SBIE_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    Sys S = sys_of(c);
    std::vector<sbie_ctx*> all = S.parts;
    if (c->is_batch) all.push_back(c);
    for (sbie_ctx* q : all) {
        q->prof.on = enable != 0;
        for (int s = 0; s < 8; ++s) {
            q->prof.ms[s] = 0;
            q->prof.launches[s] = 0;
            q->prof_used[s] = 0;
        }
        q->prof.pairs_f32 = q->prof.pairs_f64 = 0;
        q->prof.arnoldi_vectors = 0;
        q->prof.kernels0 = q->n_launch;
    }
    return SBIE_OK;
}

sbie_status sphere_bie_profile_read(sbie_ctx* c, sbie_profile* out) {
    if (!c || !out) return SBIE_ERR_ARG;
    CK(cudaStreamSynchronize(c->stream));
    std::memset(out, 0, sizeof(*out));
    Sys S = sys_of(c);
    std::vector<sbie_ctx*> all = S.parts;
    if (c->is_batch) all.push_back(c);
    for (sbie_ctx* q : all) {
        for (int s = 0; s < 8; ++s) {
            for (int i = 0; i < q->prof_used[s]; ++i) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, q->prof_events[s][i].first, q->prof_events[s][i].second));
                q->prof.ms[s] += ms;
                q->prof.launches[s] += 1;
            }
            q->prof_used[s] = 0;
            out->ms[s] += q->prof.ms[s];
            out->launches[s] += q->prof.launches[s];
        }
        out->far_pairs_f32 += q->prof.pairs_f32;
        out->far_pairs_f64 += q->prof.pairs_f64;
        out->arnoldi_vectors += q->prof.arnoldi_vectors;
        out->kernel_launches += q->n_launch - q->prof.kernels0;
    }
    return SBIE_OK;
}

sbie_status sphere_bie_solution_density(sbie_ctx* c, double* density) {
    if (!c) return SBIE_ERR_ARG;
    if (!density) return fail(c, SBIE_ERR_ARG, "NULL density");
    if (!c->has_solution) return fail(c, SBIE_ERR_ARG, "no solve has run on this context");
    CKS(to_user(c, c->d_xsol, density, true));
    CK(cudaStreamSynchronize(c->stream));
    return SBIE_OK;
}

sbie_status sphere_bie_precond_info(const sbie_ctx* c, sbie_op op, int* kind, int* n_pairs, int* n_dropped,
                                    double* setup_ms) {
    if (!c) return SBIE_ERR_ARG;
    if (op != SBIE_OP_RESISTANCE && op != SBIE_OP_MOBILITY)
        return fail(const_cast<sbie_ctx*>(c), SBIE_ERR_ARG, "the preconditioner serves the resistance and mobility operators");
    const int slot = prec_slot(op);
    int k = 0, np = 0, nd = 0;
    double ms = 0.0;
    for (const sbie_ctx* q : c->is_batch ? c->parts : std::vector<sbie_ctx*>{const_cast<sbie_ctx*>(c)}) {
        k = std::max(k, q->prec[slot].kind);
        np += q->prec[slot].n_pairs;
        nd += q->prec[slot].n_dropped;
        ms += q->prec[slot].setup_ms;
    }
    if (kind) *kind = k;
    if (n_pairs) *n_pairs = np;
    if (n_dropped) *n_dropped = nd;
    if (setup_ms) *setup_ms = ms;
    return SBIE_OK;
}

sbie_status sphere_bie_pair_network_size(long long* n_params) {
    if (!n_params) return SBIE_ERR_ARG;
    *n_params = mlp_layout().total;
    return SBIE_OK;
}

sbie_status sphere_bie_pair_blocks(int n, const double* dist, const double* a_src, const double* a_tgt, int p,
                                   sbie_op op, double* blocks) {
    if (n < 1 || !dist || !a_src || !a_tgt || !blocks || p < kPrecL || p > kMaxP ||
        (op != SBIE_OP_RESISTANCE && op != SBIE_OP_MOBILITY))
        return fail(nullptr, SBIE_ERR_ARG, "pair_blocks: bad arguments");
    for (int q = 0; q < n; ++q)
        if (!(dist[q] > a_src[q] + a_tgt[q]) || !(a_src[q] > 0) || !(a_tgt[q] > 0))
            return fail(nullptr, SBIE_ERR_ARG, "pair_blocks: spheres must be disjoint with positive radii");
    std::vector<double> out;
    CKS(aligned_blocks(n, dist, a_src, a_tgt, p, 1e9, op, out));
    std::memcpy(blocks, out.data(), sizeof(double) * out.size());
    return SBIE_OK;
}

sbie_status sphere_bie_pair_network_gradients(const float* params, int n, const float* X, const float* Y,
                                              float* grads, double* loss) {
    if (!params || !X || !Y || !grads || !loss || n < 1) return fail(nullptr, SBIE_ERR_ARG, "bad arguments");
    cudaError_t e = mlp_gradients(params, n, X, Y, grads, loss);
    if (e != cudaSuccess) return fail(nullptr, SBIE_ERR_CUDA, std::string("network gradients: ") + cudaGetErrorString(e));
    return SBIE_OK;
}

sbie_status sphere_bie_train_pair_network(const sbie_pair_train_opts* o, const char* path, sbie_pair_train_info* info) {
    if (!o || !path || o->n_samples < 16 || o->p < kPrecL || o->p > kMaxP || !(o->gap_min > 0) ||
        !(o->gap_max >= o->gap_min) || !(o->radius > 0) || o->epochs < 1 || o->batch < 1 || !(o->val_frac >= 0) ||
        !(o->val_frac < 0.9) || o->ops < 1 || o->ops > 3 || !(o->radius_max == 0.0 || o->radius_max >= o->radius))
        return fail(nullptr, SBIE_ERR_ARG, "train_pair_network: bad options");
    PairNetSet set;
    sbie_pair_train_info acc{};
    for (int op : {SBIE_OP_RESISTANCE, SBIE_OP_MOBILITY}) {
        if (!(o->ops & (op == SBIE_OP_RESISTANCE ? 1 : 2))) continue;
        PairNet net;
        sbie_pair_train_info one{};
        CKS(train_one(*o, op, net, one));
        set.nets.push_back(std::move(net));
        acc.train_loss = std::max(acc.train_loss, one.train_loss);
        acc.val_rel_err = std::max(acc.val_rel_err, one.val_rel_err);
        acc.t_data_s += one.t_data_s;
        acc.t_train_s += one.t_train_s;
        acc.n_train = one.n_train;
        acc.n_val = one.n_val;
    }
    CKS(net_save(path, set));
    if (info) *info = acc;
    return SBIE_OK;
}

}  // extern "C"
