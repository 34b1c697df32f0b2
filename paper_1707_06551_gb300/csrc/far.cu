// Far field: the smooth quadrature of Eq. 4.4 applied to the Stokeslet
// (Eq. 2.19), the double layer (Eq. 2.21, sign of Theorem 2) or the traction of
// the single layer (Eq. 2.22) over every source node of every sphere that is
// well separated from the target sphere (Eq. 4.5).  This is the dense all-pairs
// Nystrom sum; the paper hands it to an FMM.
//
// Design: one CTA owns the nodes of one target sphere (split into `chunks` if
// the sphere has more nodes than the CTA has target slots).  Source nodes are
// staged through shared memory in tiles; while staging, a source whose sphere
// is the target sphere or one of its close partners gets zero weight (a
// per-CTA bitmask over spheres), so the inner pair loop carries no mask.  The
// source range can be split over gridDim.y CTAs whose partial sums are added
// in a fixed order by far_reduce (deterministic).
//
// FP32 variant: positions are held as float hi + lo pairs and staged relative
// to the target sphere's centre, so the difference x - y keeps relative FP32
// accuracy; each tile's FP32 partial sum is added to the running total with
// Neumaier's compensated summation.
#include <algorithm>

#include "common.h"

namespace sbie {

// FP32 pair kernel layout: float4 per staged source (position, density and,
// for D, the source normal, each component duplicated) and running sums per
// target (the three components)
__host__ __device__ constexpr int f32_nv(int op) { return op == (int)Kern::D ? 5 : 3; }
__host__ __device__ constexpr int f32_na(int) { return 3; }

struct FarArgs {
    int n, npn, chunks, tile;
    long long N, split_len;
    const float4* __restrict__ xhi;
    const float4* __restrict__ xlo;
    const float4* __restrict__ nrm;
    const float4* __restrict__ srcf;
    const double4* __restrict__ x64;
    const double4* __restrict__ nrm64;
    const double4* __restrict__ src64;
    const double* __restrict__ c;
    const int* __restrict__ sph;
    const int* __restrict__ near_ptr;
    const int* __restrict__ near_idx;
    const int* __restrict__ sph_prob;  // problem of each sphere
    const int* __restrict__ prob_sph;  // first sphere of each problem (+ end)
    const int* __restrict__ live;      // per-problem flags of a running GMRES cycle, or null
    int live_off;                      // system index of this context's first problem
    double* __restrict__ part;  // [split][N][3]
};

// A target sphere whose problem stopped iterating (its Krylov vectors are
// zero): the CTA writes zero partial sums for its targets and leaves.  The
// test depends on the sphere alone, so the whole CTA takes the same branch.
__device__ __forceinline__ bool far_skip(const FarArgs& a, int sphere, int chunk, int split, int tpt) {
    if (!a.live || a.live[a.live_off + a.sph_prob[sphere]]) return false;
    double* out = a.part + (size_t)split * a.N * 3;
    for (int t = 0; t < tpt; ++t) {
        const int q = chunk * (blockDim.x * tpt) + t * blockDim.x + threadIdx.x;
        if (q >= a.npn) continue;
        const long long node = (long long)sphere * a.npn + q;
        out[node * 3] = out[node * 3 + 1] = out[node * 3 + 2] = 0.0;
    }
    return true;
}

// Source nodes of split `split` for a target sphere: its problem's nodes cut
// into gridDim.y tile-aligned pieces.
__device__ __forceinline__ void source_range(const FarArgs& a, int sphere, int split, long long& b0, long long& b1) {
    const int pr = a.sph_prob[sphere];
    const long long beg = (long long)a.prob_sph[pr] * a.npn, end = (long long)a.prob_sph[pr + 1] * a.npn;
    long long len = (end - beg + gridDim.y - 1) / gridDim.y;
    len = ((len + a.tile - 1) / a.tile) * a.tile;
    b0 = beg + (long long)split * len;
    b1 = min(end, b0 + len);
}

__device__ __forceinline__ void build_flags(const FarArgs& a, int sphere, unsigned* flags) {
    const int nw = (a.n + 31) >> 5;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) flags[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) atomicOr(&flags[sphere >> 5], 1u << (sphere & 31));
    for (int e = a.near_ptr[sphere] + threadIdx.x; e < a.near_ptr[sphere + 1]; e += blockDim.x) {
        int k = a.near_idx[e];
        atomicOr(&flags[k >> 5], 1u << (k & 31));
    }
    __syncthreads();
}

__device__ __forceinline__ void neumaier(float& sum, float& comp, float v) {
    float t = sum + v;
    if (fabsf(sum) >= fabsf(v))
        comp += (sum - t) + v;
    else
        comp += (v - t) + sum;
    sum = t;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP32 pair kernel on packed FP32x2 arithmetic: every thread owns 2 * NP
// targets held in float2 pairs, so one __ffma2_rn evaluates two (target,
// source) pairs.  Each staged source is stored pre-duplicated in shared memory
// ({-x, -x, -y, -y}, {-z, -z, fx, fx}, {fy, fy, fz, fz} and, for D, the source
// normal {nx, nx, ny, ny}, {nz, nz, 0, 0}), so every packed operand comes from
// one 128-bit shared-memory broadcast.  The compensated running sums live in
// shared memory (touched once per tile), which keeps the registers for the
// pair loop and lets more warps share each SM.
template <int OP, int NP, int MINB>
__global__ void __launch_bounds__(MINB ? 64 : 256, MINB ? MINB : 1) far_f32_kernel(FarArgs a) {
    constexpr int NV = f32_nv(OP);  // float4 per staged source
    constexpr int TPT = 2 * NP;
    const int sphere = blockIdx.x / a.chunks, chunk = blockIdx.x - sphere * a.chunks;
    const int split = blockIdx.y;
    const int tid = threadIdx.x, bd = blockDim.x;
    if (far_skip(a, sphere, chunk, split, TPT)) return;
    extern __shared__ float4 smem4[];
    // [tile][NV] staged sources | [TPT][3][2][bd] running sums and compensations | sphere flags
    float* run = reinterpret_cast<float*>(smem4 + NV * a.tile);
    unsigned* flags = reinterpret_cast<unsigned*>(run + TPT * f32_na(OP) * 2 * bd);
    build_flags(a, sphere, flags);

    const double cx = a.c[3 * sphere], cy = a.c[3 * sphere + 1], cz = a.c[3 * sphere + 2];
    const float chx = (float)cx, chy = (float)cy, chz = (float)cz;
    const float clx = (float)(cx - (double)chx), cly = (float)(cy - (double)chy), clz = (float)(cz - (double)chz);

    float2 tx[NP], ty[NP], tz[NP], tnx[NP], tny[NP], tnz[NP];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int q = chunk * (bd * TPT) + t * bd + tid;
        const long long node = (long long)sphere * a.npn + (q < a.npn ? q : a.npn - 1);
        float4 h = a.xhi[node], l = a.xlo[node];
        float px = (h.x - chx) + (l.x - clx), py = (h.y - chy) + (l.y - cly), pz = (h.z - chz) + (l.z - clz);
        float4 nn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (OP == (int)Kern::K) nn = a.nrm[node];
        if (t & 1) {
            tx[t >> 1].y = px; ty[t >> 1].y = py; tz[t >> 1].y = pz;
            tnx[t >> 1].y = nn.x; tny[t >> 1].y = nn.y; tnz[t >> 1].y = nn.z;
        } else {
            tx[t >> 1].x = px; ty[t >> 1].x = py; tz[t >> 1].x = pz;
            tnx[t >> 1].x = nn.x; tny[t >> 1].x = nn.y; tnz[t >> 1].x = nn.z;
        }
    }
#pragma unroll
    for (int e = 0; e < TPT * 6; ++e) run[e * bd + tid] = 0.f;

    long long b0, b1;
    source_range(a, sphere, split, b0, b1);
    for (long long base = b0; base < b1; base += a.tile) {
        __syncthreads();
        for (int j = tid; j < a.tile; j += bd) {
            long long s = base + j;
            float px = -1.0e4f, py = -1.0e4f, pz = -1.0e4f, fx = 0.f, fy = 0.f, fz = 0.f;
            float nx = 0.f, ny = 0.f, nz = 0.f;
            if (s < b1) {
                int k = a.sph[s];
                if (!((flags[k >> 5] >> (k & 31)) & 1u)) {
                    float4 h = a.xhi[s], l = a.xlo[s];
                    px = -((h.x - chx) + (l.x - clx));
                    py = -((h.y - chy) + (l.y - cly));
                    pz = -((h.z - chz) + (l.z - clz));
                    float4 F = a.srcf[s];
                    fx = F.x; fy = F.y; fz = F.z;
                    if (OP == (int)Kern::D) {
                        float4 nn = a.nrm[s];
                        nx = nn.x; ny = nn.y; nz = nn.z;
                    }
                }
            }
            float4* dst = smem4 + (size_t)j * NV;
            dst[0] = make_float4(px, px, py, py);
            dst[1] = make_float4(pz, pz, fx, fx);
            dst[2] = make_float4(fy, fy, fz, fz);
            if (OP == (int)Kern::D) {
                dst[3] = make_float4(nx, nx, ny, ny);
                dst[4] = make_float4(nz, nz, 0.f, 0.f);
            }
        }
        __syncthreads();
        float2 acc[NP][3];
#pragma unroll
        for (int t = 0; t < NP; ++t) acc[t][0] = acc[t][1] = acc[t][2] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int j = 0; j < a.tile; ++j) {
            const float4* src = smem4 + (size_t)j * NV;
            const float4 v0 = src[0], v1 = src[1], v2 = src[2];
            const float2 mx = make_float2(v0.x, v0.y), my = make_float2(v0.z, v0.w), mz = make_float2(v1.x, v1.y);
            const float2 fx = make_float2(v1.z, v1.w), fy = make_float2(v2.x, v2.y), fz = make_float2(v2.z, v2.w);
            float2 nx, ny, nz;
            if (OP == (int)Kern::D) {
                const float4 v3 = src[3], v4 = src[4];
                nx = make_float2(v3.x, v3.y);
                ny = make_float2(v3.z, v3.w);
                nz = make_float2(v4.x, v4.y);
            }
#pragma unroll
            for (int t = 0; t < NP; ++t) {
                const float2 dx = __fadd2_rn(tx[t], mx), dy = __fadd2_rn(ty[t], my), dz = __fadd2_rn(tz[t], mz);
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                float2 rf = __fmul2_rn(dx, fx);
                rf = __ffma2_rn(dy, fy, rf);
                rf = __ffma2_rn(dz, fz, rf);
                if (OP == (int)Kern::S) {
                    float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                    const float2 ri2 = __fmul2_rn(ri, ri);
                    const float2 s3 = __fmul2_rn(__fmul2_rn(rf, ri), ri2);
                    acc[t][0] = __ffma2_rn(dx, s3, __ffma2_rn(fx, ri, acc[t][0]));
                    acc[t][1] = __ffma2_rn(dy, s3, __ffma2_rn(fy, ri, acc[t][1]));
                    acc[t][2] = __ffma2_rn(dz, s3, __ffma2_rn(fz, ri, acc[t][2]));
                } else {
                    float2 rn;
                    if (OP == (int)Kern::D) {
                        rn = __fmul2_rn(dx, nx);
                        rn = __ffma2_rn(dy, ny, rn);
                        rn = __ffma2_rn(dz, nz, rn);
                    } else {
                        rn = __fmul2_rn(dx, tnx[t]);
                        rn = __ffma2_rn(dy, tny[t], rn);
                        rn = __ffma2_rn(dz, tnz[t], rn);
                    }
                    // r^-5 = 2^(-5/2 log2 r^2) on the special-function unit:
                    // two MUFU operations and one multiply instead of a
                    // reciprocal square root and three multiplies
                    float2 l2 = make_float2(lg2_approx(r2.x), lg2_approx(r2.y));
                    l2 = __fmul2_rn(l2, make_float2(-2.5f, -2.5f));
                    const float2 ri5 = make_float2(ex2_approx(l2.x), ex2_approx(l2.y));
                    const float2 s5 = __fmul2_rn(__fmul2_rn(rf, rn), ri5);
                    acc[t][0] = __ffma2_rn(dx, s5, acc[t][0]);
                    acc[t][1] = __ffma2_rn(dy, s5, acc[t][1]);
                    acc[t][2] = __ffma2_rn(dz, s5, acc[t][2]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < NP; ++t)
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float* sp = run + (((2 * t + h) * 3 + d) * 2) * bd + tid;
                    float sm = sp[0], cm = sp[bd];
                    neumaier(sm, cm, h ? acc[t][d].y : acc[t][d].x);
                    sp[0] = sm;
                    sp[bd] = cm;
                }
    }
    double* out = a.part + (size_t)split * a.N * 3;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int q = chunk * (bd * TPT) + t * bd + tid;
        if (q >= a.npn) continue;
        const long long node = (long long)sphere * a.npn + q;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float* sp = run + ((t * 3 + d) * 2) * bd + tid;
            out[node * 3 + d] = (double)sp[0] + (double)sp[bd];
        }
    }
}

// ---- double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two floats.  Building blocks: Knuth's TwoSum, Dekker's Fast2Sum and the
// FMA-based exact product; about 48 significant bits.
struct df {
    float h, l;
};
__device__ __forceinline__ df df_split(double x) {
    float h = (float)x;
    return df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = a + b;
    return df{s, b - (s - a)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return df{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_sub(df x, df y) {  // x - y
    df s = two_sum(x.h, -y.h);
    s.l += x.l - y.l;
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.h, y.h);
    s.l += x.l + y.l;
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ df df_mul(df x, df y) {
    float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_sqr(df x) {
    float p = x.h * x.h;
    float e = fmaf(x.h, x.h, -p);
    e = fmaf(2.f * x.h, x.l, e);
    return fast_two_sum(p, e);
}
// Lighter building blocks for the pair loop.  A product of two normalised
// values is left as (p, e) with |e| <= ulp(p) (no renormalisation: the next
// product or sum absorbs it); a difference keeps the exact TwoSum high part.
__device__ __forceinline__ df df_diff(df x, df y) {  // x - y
    df s = two_sum(x.h, -y.h);
    return df{s.h, s.l + (x.l - y.l)};
}
__device__ __forceinline__ df df_mul_l(df x, df y) {
    float p = x.h * y.h;
    float e = fmaf(x.h, y.h, -p);
    e = fmaf(x.h, y.l, e);
    e = fmaf(x.l, y.h, e);
    return df{p, e};
}
__device__ __forceinline__ df df_sqr_l(df x) {
    float p = x.h * x.h;
    float e = fmaf(x.h, x.h, -p);
    e = fmaf(x.h + x.h, x.l, e);
    return df{p, e};
}
// sum of three such (p, e) terms, renormalised (the sum may cancel)
__device__ __forceinline__ df df_sum3(df a, df b, df c) {
    df s = two_sum(a.h, b.h);
    df t = two_sum(s.h, c.h);
    return two_sum(t.h, (s.l + t.l) + (a.l + b.l + c.l));
}

// 1/sqrt(x) for x > 0: hardware estimate y0, then one Newton step carried in
// df with its second-order term: y = y0 (1 - t/2 + 3 t^2 / 8), t = x y0^2 - 1.
__device__ __forceinline__ df df_rsqrt(df x) {
    float y0 = rsqrt_approx(x.h);
    float q = y0 * y0;
    float ql = fmaf(y0, y0, -q);
    float h = x.h * q;
    float e = fmaf(x.h, q, -h);
    e = fmaf(x.h, ql, e);
    e = fmaf(x.l, q, e);
    float t = (h - 1.0f) + e;
    float corr = y0 * t * fmaf(0.375f, t, -0.5f);
    return fast_two_sum(y0, corr);
}

// Far field with every pair evaluated in df arithmetic (about 1e-13 relative
// per pair), sums within a tile in df and across tiles in FP64.  Sources are
// staged relative to the target sphere's centre, computed in FP64 and split.
template <int OP>
__global__ void __launch_bounds__(256) far_df_kernel(FarArgs a) {
    constexpr int NV = (OP == (int)Kern::D) ? 5 : 3;  // float4 per staged source: pos(6) dens(6) [nrm(6)]
    const int sphere = blockIdx.x / a.chunks, chunk = blockIdx.x - sphere * a.chunks;
    const int split = blockIdx.y;
    const int tid = threadIdx.x, bd = blockDim.x;
    if (far_skip(a, sphere, chunk, split, 1)) return;
    extern __shared__ float4 smem4[];
    unsigned* flags = reinterpret_cast<unsigned*>(smem4 + NV * a.tile);
    build_flags(a, sphere, flags);
    const double cx = a.c[3 * sphere], cy = a.c[3 * sphere + 1], cz = a.c[3 * sphere + 2];
    const int q = chunk * bd + tid;
    const bool tval = q < a.npn;
    const long long tnode = (long long)sphere * a.npn + (tval ? q : a.npn - 1);
    const double4 X = a.x64[tnode];
    const df tx = df_split(X.x - cx), ty = df_split(X.y - cy), tz = df_split(X.z - cz);
    df tnx{0.f, 0.f}, tny{0.f, 0.f}, tnz{0.f, 0.f};
    if (OP == (int)Kern::K) {
        const double4 nn = a.nrm64[tnode];
        tnx = df_split(nn.x); tny = df_split(nn.y); tnz = df_split(nn.z);
    }
    double sum[3] = {0.0, 0.0, 0.0};
    long long b0, b1;
    source_range(a, sphere, split, b0, b1);
    for (long long base = b0; base < b1; base += a.tile) {
        __syncthreads();
        for (int j = tid; j < a.tile; j += bd) {
            long long s = base + j;
            double px = 1.0e4, py = 1.0e4, pz = 1.0e4, fx = 0, fy = 0, fz = 0, nx = 0, ny = 0, nz = 0;
            if (s < b1) {
                int k = a.sph[s];
                if (!((flags[k >> 5] >> (k & 31)) & 1u)) {
                    const double4 P = a.x64[s];
                    px = P.x - cx; py = P.y - cy; pz = P.z - cz;
                    const double4 F = a.src64[s];
                    fx = F.x; fy = F.y; fz = F.z;
                    if (OP == (int)Kern::D) {
                        const double4 nn = a.nrm64[s];
                        nx = nn.x; ny = nn.y; nz = nn.z;
                    }
                }
            }
            const df qx = df_split(px), qy = df_split(py), qz = df_split(pz);
            const df gx = df_split(fx), gy = df_split(fy), gz = df_split(fz);
            float4* dst = smem4 + (size_t)j * NV;
            dst[0] = make_float4(qx.h, qx.l, qy.h, qy.l);
            dst[1] = make_float4(qz.h, qz.l, gx.h, gx.l);
            dst[2] = make_float4(gy.h, gy.l, gz.h, gz.l);
            if (OP == (int)Kern::D) {
                const df mx = df_split(nx), my = df_split(ny), mz = df_split(nz);
                dst[3] = make_float4(mx.h, mx.l, my.h, my.l);
                dst[4] = make_float4(mz.h, mz.l, 0.f, 0.f);
            }
        }
        __syncthreads();
        df acc0{0.f, 0.f}, acc1{0.f, 0.f}, acc2{0.f, 0.f};
#pragma unroll 2
        for (int j = 0; j < a.tile; ++j) {
            const float4* src = smem4 + (size_t)j * NV;
            const float4 v0 = src[0], v1 = src[1], v2 = src[2];
            const df dx = df_diff(tx, df{v0.x, v0.y}), dy = df_diff(ty, df{v0.z, v0.w}), dz = df_diff(tz, df{v1.x, v1.y});
            const df fx{v1.z, v1.w}, fy{v2.x, v2.y}, fz{v2.z, v2.w};
            // |d|^2 and the dot products: exact products, one renormalised sum
            const df q = df_sum3(df_sqr_l(dx), df_sqr_l(dy), df_sqr_l(dz));
            const df ri = df_rsqrt(q);
            const df ri2 = df_sqr_l(ri);
            const df rf = df_sum3(df_mul_l(dx, fx), df_mul_l(dy, fy), df_mul_l(dz, fz));
            if (OP == (int)Kern::S) {
                const df s3 = df_mul_l(df_mul_l(rf, ri), ri2);
                const df ax = df_add(df_mul_l(fx, ri), df_mul_l(dx, s3));
                const df ay = df_add(df_mul_l(fy, ri), df_mul_l(dy, s3));
                const df az = df_add(df_mul_l(fz, ri), df_mul_l(dz, s3));
                df t = two_sum(acc0.h, ax.h); acc0 = df{t.h, acc0.l + (t.l + ax.l)};
                t = two_sum(acc1.h, ay.h); acc1 = df{t.h, acc1.l + (t.l + ay.l)};
                t = two_sum(acc2.h, az.h); acc2 = df{t.h, acc2.l + (t.l + az.l)};
            } else {
                df rn;
                if (OP == (int)Kern::D) {
                    const float4 v3 = src[3], v4 = src[4];
                    rn = df_sum3(df_mul_l(dx, df{v3.x, v3.y}), df_mul_l(dy, df{v3.z, v3.w}), df_mul_l(dz, df{v4.x, v4.y}));
                } else {
                    rn = df_sum3(df_mul_l(dx, tnx), df_mul_l(dy, tny), df_mul_l(dz, tnz));
                }
                const df s5 = df_mul_l(df_mul_l(rf, rn), df_mul_l(df_sqr_l(ri2), ri));
                // running sums: exact TwoSum of the high parts, low parts
                // gathered and renormalised once per tile
                const df ax = df_mul_l(dx, s5), ay = df_mul_l(dy, s5), az = df_mul_l(dz, s5);
                df t = two_sum(acc0.h, ax.h); acc0 = df{t.h, acc0.l + (t.l + ax.l)};
                t = two_sum(acc1.h, ay.h); acc1 = df{t.h, acc1.l + (t.l + ay.l)};
                t = two_sum(acc2.h, az.h); acc2 = df{t.h, acc2.l + (t.l + az.l)};
            }
        }
        sum[0] += (double)acc0.h + (double)acc0.l;
        sum[1] += (double)acc1.h + (double)acc1.l;
        sum[2] += (double)acc2.h + (double)acc2.l;
    }
    if (tval) {
        double* out = a.part + (size_t)split * a.N * 3;
        for (int d = 0; d < 3; ++d) out[tnode * 3 + d] = sum[d];
    }
}

template <int OP, int TPT>
__global__ void __launch_bounds__(256) far_f64_kernel(FarArgs a) {
    constexpr int NV = (OP == (int)Kern::D) ? 3 : 2;
    const int sphere = blockIdx.x / a.chunks, chunk = blockIdx.x - sphere * a.chunks;
    const int split = blockIdx.y;
    const int tid = threadIdx.x, bd = blockDim.x;
    if (far_skip(a, sphere, chunk, split, TPT)) return;
    extern __shared__ double4 smem8[];
    double4* s_pos = smem8;
    double4* s_den = smem8 + a.tile;
    double4* s_nrm = smem8 + 2 * a.tile;
    unsigned* flags = reinterpret_cast<unsigned*>(smem8 + NV * a.tile);
    build_flags(a, sphere, flags);

    double tx[TPT], ty[TPT], tz[TPT], tnx[TPT], tny[TPT], tnz[TPT];
    long long tnode[TPT];
    bool tval[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        int q = chunk * (bd * TPT) + t * bd + tid;
        tval[t] = q < a.npn;
        long long node = (long long)sphere * a.npn + (tval[t] ? q : a.npn - 1);
        tnode[t] = node;
        double4 x = a.x64[node];
        tx[t] = x.x; ty[t] = x.y; tz[t] = x.z;
        if (OP == (int)Kern::K) {
            double4 nn = a.nrm64[node];
            tnx[t] = nn.x; tny[t] = nn.y; tnz[t] = nn.z;
        } else {
            tnx[t] = tny[t] = tnz[t] = 0.0;
        }
    }
    double acc[TPT][3];
#pragma unroll
    for (int t = 0; t < TPT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = 0.0;
    const double far_off = 1.0e6;
    long long b0, b1;
    source_range(a, sphere, split, b0, b1);
    for (long long base = b0; base < b1; base += a.tile) {
        __syncthreads();
        for (int j = tid; j < a.tile; j += bd) {
            long long s = base + j;
            double4 P = make_double4(tx[0] + far_off, ty[0] + far_off, tz[0] + far_off, 0.0);
            double4 F = make_double4(0, 0, 0, 0), Nn = make_double4(0, 0, 0, 0);
            if (s < b1) {
                int k = a.sph[s];
                if (!((flags[k >> 5] >> (k & 31)) & 1u)) {
                    P = a.x64[s];
                    F = a.src64[s];
                    if (OP == (int)Kern::D) Nn = a.nrm64[s];
                }
            }
            s_pos[j] = P;
            s_den[j] = F;
            if (OP == (int)Kern::D) s_nrm[j] = Nn;
        }
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < a.tile; ++j) {
            const double4 P = s_pos[j];
            const double4 F = s_den[j];
            double4 Nn;
            if (OP == (int)Kern::D) Nn = s_nrm[j];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                double dx = tx[t] - P.x, dy = ty[t] - P.y, dz = tz[t] - P.z;
                double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
                double ri = rsqrt(r2);
                double ri2 = ri * ri;
                double rf = fma(dz, F.z, fma(dy, F.y, dx * F.x));
                if (OP == (int)Kern::S) {
                    double s3 = rf * ri * ri2;
                    acc[t][0] = fma(dx, s3, fma(F.x, ri, acc[t][0]));
                    acc[t][1] = fma(dy, s3, fma(F.y, ri, acc[t][1]));
                    acc[t][2] = fma(dz, s3, fma(F.z, ri, acc[t][2]));
                } else {
                    double rn;
                    if (OP == (int)Kern::D)
                        rn = fma(dz, Nn.z, fma(dy, Nn.y, dx * Nn.x));
                    else
                        rn = fma(dz, tnz[t], fma(dy, tny[t], dx * tnx[t]));
                    double s5 = (rf * rn) * (ri2 * ri2) * ri;
                    acc[t][0] = fma(dx, s5, acc[t][0]);
                    acc[t][1] = fma(dy, s5, acc[t][1]);
                    acc[t][2] = fma(dz, s5, acc[t][2]);
                }
            }
        }
    }
    double* out = a.part + (size_t)split * a.N * 3;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        if (!tval[t]) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) out[tnode[t] * 3 + d] = acc[t][d];
    }
}

// out[i] = scale * sum_k part[k][i] for the first `count` entries of partials
// laid out [split][stride]
__global__ void far_reduce(const double* __restrict__ part, int split, long long stride, long long count,
                           double scale, int accumulate, double* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s = 0.0;
    for (int k = 0; k < split; ++k) s += part[(size_t)k * stride + i];
    out[i] = accumulate ? out[i] + scale * s : scale * s;
}

__global__ void pack_kernel(const double* __restrict__ dens, const double* __restrict__ x64, long long N,
                            float4* __restrict__ srcf, double4* __restrict__ src64) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double w = x64[4 * i + 3];
    double fx = dens[3 * i] * w, fy = dens[3 * i + 1] * w, fz = dens[3 * i + 2] * w;
    if (srcf) srcf[i] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
    if (src64) src64[i] = make_double4(fx, fy, fz, 0.0);
}

cudaError_t launch_pack(sbie_ctx* c, const double* dens, int mode) {
    int th = 256;
    long long blocks = (c->N + th - 1) / th;
    const bool f32 = mode == kModeF32;
    pack_kernel<<<(unsigned)blocks, th, 0, c->stream>>>(dens, c->d_x, c->N, f32 ? c->d_srcf : nullptr,
                                                        f32 ? nullptr : c->d_src64); ++c->n_launch;
    return cudaGetLastError();
}

long long far_pairs(const sbie_ctx* c) {
    long long tot = 0;
    for (int pr = 0; pr < c->n_prob; ++pr) {
        const long long nodes = (long long)(c->h_prob_sph[pr + 1] - c->h_prob_sph[pr]) * c->npn;
        for (int i = c->h_prob_sph[pr]; i < c->h_prob_sph[pr + 1]; ++i) {
            long long excl = 1 + (c->h_near_ptr[i + 1] - c->h_near_ptr[i]);
            tot += (long long)c->npn * (nodes - excl * c->npn);
        }
    }
    return tot;
}

// nts: target spheres launched (the first nts; all of them outside timing)
template <int OP>
static cudaError_t launch_far_df(sbie_ctx* c, const FarTune& tu, const FarArgs& a, int nts) {
    dim3 grid(nts * a.chunks, tu.split);
    const int nv = (OP == (int)Kern::D) ? 5 : 3;
    size_t sm = (size_t)nv * tu.tile * sizeof(float4) + ((c->n + 31) / 32) * sizeof(unsigned);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(far_df_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    far_df_kernel<OP><<<grid, tu.threads, sm, c->stream>>>(a); ++c->n_launch;
    return cudaGetLastError();
}

// Dynamic shared memory of the FP32 pair kernel: staged sources, the running
// sums with their compensations for every target of a thread, sphere flags.
template <int OP>
static size_t f32_smem(int tpt, int threads, int tile, int n) {
    return (size_t)f32_nv(OP) * tile * sizeof(float4) +
           (size_t)2 * ((tpt + 1) / 2) * f32_na(OP) * 2 * threads * sizeof(float) + ((n + 31) / 32) * sizeof(unsigned);
}

// The FP32 pair kernel is compiled once without a register cap (about 150-210
// registers for 4-6 targets per thread) and, for 64-thread CTAs, with 8, 10 and
// 16 resident CTAs per SM required (about 128, 96 and 64 registers: 4, 5 and 8
// warps per scheduler).
// Fewer registers mean more warps to hide the special-function and FMA
// latencies but more register moves; the autotuner times each build.
using F32Kernel = void (*)(FarArgs);
template <int OP, int NP>
static F32Kernel f32_build(const FarTune& tu) {
    if (tu.threads != 64) return far_f32_kernel<OP, NP, 0>;
    switch (tu.minb) {
        case 8: return far_f32_kernel<OP, NP, 8>;
        case 10: return far_f32_kernel<OP, NP, 10>;
        case 16: return far_f32_kernel<OP, NP, 16>;
        default: return far_f32_kernel<OP, NP, 0>;
    }
}
// The builds the autotuner times for `tpt` targets per thread: capping two
// targets per thread (94 registers uncapped) only matters at 64 registers.
int far_f32_builds(int tpt, int* minb) {
    if (tpt <= 2) { minb[0] = 0; minb[1] = 16; return 2; }
    minb[0] = 0; minb[1] = 8; minb[2] = 10; minb[3] = 16;
    return 4;
}

template <int OP, int TPT>
static cudaError_t launch_far_t(sbie_ctx* c, const FarTune& tu, bool f32, const FarArgs& a, int nts) {
    dim3 grid(nts * a.chunks, tu.split);
    int nv = (OP == (int)Kern::D) ? 3 : 2;
    size_t words = ((c->n + 31) / 32) * sizeof(unsigned);
    if (f32) {
        const size_t sm = f32_smem<OP>(TPT, tu.threads, tu.tile, c->n);
        auto run = [&](auto kernel) {
            if (sm > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e != cudaSuccess) return e;
            }
            kernel<<<grid, tu.threads, sm, c->stream>>>(a);
            ++c->n_launch;
            return cudaSuccess;
        };
        cudaError_t e = run(f32_build<OP, (TPT + 1) / 2>(tu));
        if (e != cudaSuccess) return e;
    } else if constexpr (TPT <= 4) {  // the FP64 kernel holds at most 4 targets per thread
        size_t sm = (size_t)nv * tu.tile * sizeof(double4) + words;
        if (sm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(far_f64_kernel<OP, TPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        far_f64_kernel<OP, TPT><<<grid, tu.threads, sm, c->stream>>>(a); ++c->n_launch;
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int OP>
static cudaError_t launch_far_op(sbie_ctx* c, const FarTune& tu, bool f32, const FarArgs& a, int nts) {
    switch (tu.tpt) {
        case 1: return launch_far_t<OP, 1>(c, tu, f32, a, nts);
        case 2: return launch_far_t<OP, 2>(c, tu, f32, a, nts);
        case 6: return f32 ? launch_far_t<OP, 6>(c, tu, true, a, nts) : cudaErrorInvalidValue;
        default: return launch_far_t<OP, 4>(c, tu, f32, a, nts);
    }
}

static FarArgs make_args(sbie_ctx* c, const FarTune& tu) {
    FarArgs a;
    a.n = c->n;
    a.npn = c->npn;
    a.N = c->N;
    a.tile = tu.tile;
    a.chunks = (c->npn + tu.threads * tu.tpt - 1) / (tu.threads * tu.tpt);
    long long per = (c->N + tu.split - 1) / tu.split;
    a.split_len = ((per + tu.tile - 1) / tu.tile) * tu.tile;
    a.xhi = c->d_xhi; a.xlo = c->d_xlo; a.nrm = c->d_nrm; a.srcf = c->d_srcf;
    a.x64 = reinterpret_cast<const double4*>(c->d_x);
    a.nrm64 = reinterpret_cast<const double4*>(c->d_nrm64);
    a.src64 = c->d_src64;
    a.c = c->d_c; a.sph = c->d_sph; a.near_ptr = c->d_near_ptr; a.near_idx = c->d_near_idx;
    a.sph_prob = c->d_sph_prob; a.prob_sph = c->d_prob_sph;
    a.part = c->d_part;
    a.live = c->far_live;
    a.live_off = c->far_live_off;
    return a;
}

static cudaError_t launch_pair_kernel(sbie_ctx* c, Kern op, int mode, const FarTune& tu, int nts) {
    FarArgs a = make_args(c, tu);
    if (mode == kModeDF) {
        switch (op) {
            case Kern::S: return launch_far_df<(int)Kern::S>(c, tu, a, nts);
            case Kern::D: return launch_far_df<(int)Kern::D>(c, tu, a, nts);
            default: return launch_far_df<(int)Kern::K>(c, tu, a, nts);
        }
    }
    const bool f32 = mode == kModeF32;
    switch (op) {
        case Kern::S: return launch_far_op<(int)Kern::S>(c, tu, f32, a, nts);
        case Kern::D: return launch_far_op<(int)Kern::D>(c, tu, f32, a, nts);
        default: return launch_far_op<(int)Kern::K>(c, tu, f32, a, nts);
    }
}

cudaError_t launch_far(sbie_ctx* c, Kern op, int mode, double* out, bool accumulate) {
    const FarTune& tu = mode == kModeF32 ? c->tune32[(int)op] : (mode == kModeDF ? c->tunedf[(int)op] : c->tune64[(int)op]);
    cudaError_t e;
    {
        StageScope st(c, mode == kModeF32 ? ST_FARK32 : ST_FARK64);
        e = launch_pair_kernel(c, op, mode, tu, c->n);
    }
    if (e != cudaSuccess) return e;
    double scale = (op == Kern::S) ? 1.0 / (8.0 * kPi) : (op == Kern::D ? 3.0 / (4.0 * kPi) : -3.0 / (4.0 * kPi));
    long long n3 = c->N * 3;
    far_reduce<<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>(c->d_part, tu.split, n3, n3, scale,
                                                                     accumulate ? 1 : 0, out); ++c->n_launch;
    return cudaGetLastError();
}

// Resident CTAs per SM of the pair kernel for tiling `tu` (registers and
// shared memory of that instantiation), or 0 if it cannot be queried.
template <typename K>
static int occ_of(K kernel, int threads, size_t sm) {
    int blocks = 0;
    if (sm > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, sm) != cudaSuccess) return 0;
    return blocks;
}

template <int OP>
static int far_occupancy_op(sbie_ctx* c, int mode, const FarTune& tu) {
    const size_t words = ((c->n + 31) / 32) * sizeof(unsigned);
    if (mode == kModeDF) {
        const int nv = (OP == (int)Kern::D) ? 5 : 3;
        return occ_of(far_df_kernel<OP>, tu.threads, (size_t)nv * tu.tile * sizeof(float4) + words);
    }
    const size_t sm = f32_smem<OP>(tu.tpt, tu.threads, tu.tile, c->n);
    switch (tu.tpt) {
        case 2: return occ_of(f32_build<OP, 1>(tu), tu.threads, sm);
        case 6: return occ_of(f32_build<OP, 3>(tu), tu.threads, sm);
        default: return occ_of(f32_build<OP, 2>(tu), tu.threads, sm);
    }
}

int far_occupancy(sbie_ctx* c, Kern op, int mode, const FarTune& tu) {
    if (mode == kModeF64) return 0;
    switch (op) {
        case Kern::S: return far_occupancy_op<(int)Kern::S>(c, mode, tu);
        case Kern::D: return far_occupancy_op<(int)Kern::D>(c, mode, tu);
        default: return far_occupancy_op<(int)Kern::K>(c, mode, tu);
    }
}

// One pair-kernel launch and the reduction of its partial sums, timed with
// CUDA events (a larger split costs the reduction more).  Large contexts time
// the first 512 target spheres only (every CTA does the same work as in a full
// launch, and 512 spheres are several waves), so tuning stays cheap.  The
// reduction writes into the partial-sum slot after the last one read, which
// the caller provides (capacity for split + 1 slots).
cudaError_t time_far(sbie_ctx* c, Kern op, int mode, const FarTune& tu, float* ms) {
    const long long n3 = c->N * 3;
    if ((size_t)(tu.split + 1) * (size_t)n3 > c->part_cap) return cudaErrorInvalidValue;
    const int nts = std::min(c->n, 512);
    const long long count = (long long)nts * c->npn * 3;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    e = cudaEventRecord(e0, c->stream);
    if (e == cudaSuccess) e = launch_pair_kernel(c, op, mode, tu, nts);
    if (e == cudaSuccess) {
        far_reduce<<<(unsigned)((count + 255) / 256), 256, 0, c->stream>>>(c->d_part, tu.split, n3, count, 1.0, 0,
                                                                         c->d_part + (size_t)tu.split * n3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace sbie
