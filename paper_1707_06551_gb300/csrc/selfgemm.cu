// Self term of the FP32 operator as one dense GEMM on the tensor cores.
//
// The self interaction of a sphere (Sec. 4.1, Eqs. 4.6-4.7) -- VSH analysis
// (Eqs. 2.12-2.14: DFT in phi, Gauss-Legendre contraction in theta), the
// Theorem 2 signature, synthesis (Eqs. 2.15-2.17) -- is a fixed linear map of
// the sphere's 3 npn nodal density values, the same for every sphere of one
// order p (the single layer scales by the radius, Theorem 2 being stated for
// the unit sphere; the double layer and the traction are scale free and share
// one principal-value signature).  So the transform contraction of every
// sphere of a context is one GEMM
//     out[:, s] (+)= scale_s * M x_s,     M: (3 npn) x (3 npn),
// with M probed once, column by column, by the FP64 self kernel applied to
// unit densities.  The pair preconditioner's H (1/D+ above degree 4, 2 on the
// rest) is a third such matrix, with the 73 low-mode analysis rows (degree <= 4
// coefficients) appended so that one GEMM also gives the coarse correction's
// input.
//
// Arithmetic: 3xTF32 -- each operand split into a TF32 high part and a TF32
// remainder, C = Ah Bh + Ah Bl + Al Bh accumulated in FP32 in tensor memory --
// which carries the contraction to about 2^-21 relative, the accuracy of the
// rest of the FP32 operator.  FP64 stays with the close-pair coefficients and
// with the FP64-accurate operator of the residuals, which keep the FP64
// transform of self.cu.
//
// Kernel (sm_103a): one CTA computes a 128 (matrix rows) x 64 (spheres) tile.
// Warp 0 lane 0 streams the four operand tiles of each K block (32 TF32 values
// = one 128-byte swizzle span) with TMA into a 4-deep shared-memory ring;
// warp 1 lane 0 issues tcgen05.mma (M = 128, N = 64, K = 8, twelve per K
// block) into 64-column TMEM accumulators and releases each ring slot with
// tcgen05.commit; all four warps then read the accumulators with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = matrix rows) and write the FP64
// output, coalesced along the matrix rows (= the nodal components of one
// sphere).  Every mbarrier wait is bounded in time; a wait that runs out
// records an error flag that the host turns into a failed launch.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "common.h"
#include "mlp.h"

namespace sbie {

namespace {

constexpr int kBM = 128;           // matrix rows per CTA (TMEM lanes)
constexpr int kBN = 64;            // spheres per CTA (TMEM columns, MMA N)
// The tensor core rounds each MMA's FP32 result toward zero, so a long chain
// of accumulations into one TMEM accumulator drifts low (measured: 5e-6
// relative after the 92 high-part MMAs of K = 726).  The high-part products
// therefore rotate over kAcc accumulators (K block kb into kb mod kAcc) and
// the two small cross products, 2^-11 of the result, share one more; the
// epilogue adds them in FP64.
constexpr int kAcc = 7;
constexpr int kTmemCols = 512;     // (kAcc + 1) x kBN, a power of two
constexpr int kBK = 32;            // K per stage: 32 fp32 = 128 bytes
constexpr int kStages = 4;
constexpr int kTileA = kBM * kBK * 4;   // bytes of one A tile (hi or lo)
constexpr int kTileB = kBN * kBK * 4;   // bytes of one B tile
constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

static_assert((kAcc + 1) * kBN <= kTmemCols, "accumulators exceed the TMEM allocation");
static_assert(kStageBytes % 1024 == 0, "stages must keep the 1024-byte alignment of 128-byte swizzled tiles");

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Waits for the phase of the given parity to complete; false if it has not
// after kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(
            tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// float -> double through the bit pattern (integer pipe): exact for normal
// numbers, zero for zero and subnormals, infinities and NaN kept.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    unsigned long long d = (unsigned long long)(u & 0x80000000u) << 32;
    if (e != 0) {
        const unsigned long long de = e == 0xFFu ? 2047ull : (unsigned long long)(e + 896u);
        d |= (de << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
    }
    return __longlong_as_double((long long)d);
}

struct GemmEpi {
    int rows;            // matrix rows with an output
    int out_rows;        // rows written to `out` (the nodal components); rows above go to `low`
    int cols;            // spheres
    long long ld_out;    // doubles between consecutive spheres of `out` (3 npn)
    double* out;
    int accumulate;      // out += instead of out =
    const float* scale;  // per-sphere factor (single layer: the radius) or nullptr
    double* low;         // [cols][rows - out_rows] or nullptr
    int k_blocks;
    int k_total;         // K blocks of the whole product (= k_blocks: no split)
    int exact;           // bit 0: A, bit 1: B has no TF32 remainder (neither loaded nor multiplied)
    int* err;            // set to 1 when a wait runs out
};

// Epilogue of the pair network's GEMMs, stored transposed so that the TMEM
// lanes (m) are the contiguous index: C[n ldc + m] = acc (+ bias[m]) (tanh)
// (x (1 - G[n ldg + m]^2)), FP32, m < M, n < N.
struct MlpEpi {
    int M, N;
    long long ldc, ldg;
    float* C;
    const float* bias;
    const float* G;
    int mode;            // TcEpi::Mode
    int k_blocks;        // K blocks of one CTA (a split-K slice when gridDim.z > 1)
    int k_total;         // K blocks of the whole product (the last slice may be shorter)
    int exact;
    int* err;
    long long zstride;   // split K: slice z writes raw sums to C + z zstride
};

template <typename EP>
__global__ void __launch_bounds__(128, 1)
    self_gemm_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                     EP E) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kStages];
    __shared__ __align__(8) uint64_t empty_bar[kStages];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const uint32_t base = (smem_addr(smem_raw) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_addr(&full_bar[s]), 1);
            mbar_init(smem_addr(&empty_bar[s]), 1);
        }
        mbar_init(smem_addr(&done_bar), 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int kb0 = blockIdx.z * E.k_blocks;  // first K block of this CTA (split K)
    const int nk = min(E.k_blocks, E.k_total - kb0);
    int issued = 0;  // K blocks whose copies the producer started

    if (warp == 0 && lane == 0) {
        // producer: TMA of the four tiles of each K block into the ring
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !mbar_wait(smem_addr(&empty_bar[s]), ((kb / kStages) + 1) & 1)) {
                failed = 1;
                break;
            }
            const uint32_t st = base + s * kStageBytes;
            const uint32_t fb = smem_addr(&full_bar[s]);
            const bool xa = !(E.exact & 1), xb = !(E.exact & 2);  // remainders present
            mbar_expect_tx(fb, kTileA + kTileB + (xa ? kTileA : 0) + (xb ? kTileB : 0));
            const int kx = (kb0 + kb) * kBK;
            tma_load_2d(st, &tmAh, kx, m0, fb);
            if (xa) tma_load_2d(st + kTileA, &tmAl, kx, m0, fb);
            tma_load_2d(st + 2 * kTileA, &tmBh, kx, n0, fb);
            if (xb) tma_load_2d(st + 2 * kTileA + kTileB, &tmBl, kx, n0, fb);
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: C = Ah Bh + Ah Bl + Al Bh, K = 8 per instruction
        constexpr uint32_t idesc = tf32_idesc(kBM, kBN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(smem_addr(&full_bar[s]), (kb / kStages) & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * kStageBytes;
#pragma unroll
            for (int kk = 0; kk < kBK / 8; ++kk) {
                const uint32_t off = kk * 32;  // 8 TF32 values
                const uint64_t ah = sw128_desc(st + off), al = sw128_desc(st + kTileA + off);
                const uint64_t bh = sw128_desc(st + 2 * kTileA + off), bl = sw128_desc(st + 2 * kTileA + kTileB + off);
                const uint32_t dj = tmem + (uint32_t)((kb % kAcc) * kBN), de = tmem + (uint32_t)(kAcc * kBN);
                mma_tf32(dj, ah, bh, idesc, (kb >= kAcc || kk > 0) ? 1u : 0u);
                bool first = (kb | kk) == 0;  // first cross product: overwrite the accumulator
                if (!(E.exact & 2)) {
                    mma_tf32(de, ah, bl, idesc, first ? 0u : 1u);
                    first = false;
                }
                if (!(E.exact & 1)) mma_tf32(de, al, bh, idesc, first ? 0u : 1u);
            }
            mma_commit(smem_addr(&empty_bar[s]));
        }
        if (!ok) failed = 1;
        mma_commit(smem_addr(&done_bar));
    }
    __syncwarp();

    // epilogue: all warps wait for the accumulator
    bool ok = mbar_wait(smem_addr(&done_bar), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok || failed) {
        if (threadIdx.x == 0) atomicExch(E.err, 1);
        // let the copies still in flight land before the CTA exits (bounded):
        // the last phase started on each ring slot
        if (warp == 0 && lane == 0)
            for (int kb = issued > kStages ? issued - kStages : 0; kb < issued; ++kb)
                (void)mbar_wait(smem_addr(&full_bar[kb % kStages]), (kb / kStages) & 1);
    } else {
        const int r = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const int used = nk < kAcc ? nk : kAcc;  // accumulators written
        // The SM issues FP64 at a small fraction of its FP32 rate, so the
        // epilogue stays in FP32 and integer arithmetic: the accumulators are
        // added in FP32 (round to nearest: no drift; the result carries FP32
        // accuracy, as the rest of the FP32 operator), the radius applied in
        // FP32, and the value widened to FP64 by its bit pattern.  Only
        // `accumulate` costs one FP64 add per output.
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 16) {
            float acc[16];
            float v[16];
            tmem_ld16(trow + (uint32_t)(kAcc * kBN + c0), acc);
#pragma unroll 1
            for (int j = 0; j < used; ++j) {
                tmem_ld16(trow + (uint32_t)(j * kBN + c0), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] += v[i];
            }
            if constexpr (std::is_same<EP, GemmEpi>::value) {
                if (r < E.rows) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int s = n0 + c0 + i;
                        if (s >= E.cols) break;
                        const double x = widen(E.scale ? acc[i] * E.scale[s] : acc[i]);
                        if (r < E.out_rows) {
                            double* o = E.out + (long long)s * E.ld_out + r;
                            *o = E.accumulate ? *o + x : x;
                        } else {
                            E.low[(long long)s * (E.rows - E.out_rows) + (r - E.out_rows)] = x;
                        }
                    }
                }
            } else {
                if (r < E.M) {
                    float* C = E.C + blockIdx.z * E.zstride;
                    const float b = (E.mode == TcEpi::kBias || E.mode == TcEpi::kBiasTanh) ? E.bias[r] : 0.f;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int n = n0 + c0 + i;
                        if (n >= E.N) break;
                        float v = acc[i] + b;
                        if (E.mode == TcEpi::kBiasTanh) v = tanhf(v);
                        if (E.mode == TcEpi::kDTanh) {
                            const float gv = E.G[(long long)n * E.ldg + r];
                            v *= 1.f - gv * gv;
                        }
                        C[(long long)n * E.ldc + r] = v;  // the warp's 32 lanes: 32 consecutive m
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// rows of src (FP64, row r at src + r * ld) -> TF32 hi / remainder pairs [rows][Kpad] (zero past K)
__global__ void split_rows_kernel(const double* __restrict__ src, long long ld, int rows, int K, int Kpad,
                                  float* __restrict__ hi, float* __restrict__ lo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * Kpad) return;
    const long long r = i / Kpad;
    const int k = (int)(i - r * Kpad);
    float h = 0.f, l = 0.f;
    if (k < K) {
        const double v = src[r * ld + k];
        h = tf32_hi((float)v);
        l = (float)(v - (double)h);
    }
    hi[i] = h;
    lo[i] = l;
}

// probe columns -> matrix rows: M[r][k] = probe[k][r] (+ diag on r == k); rows
// out_rows.. from the low-mode coefficients of each probe column
__global__ void probe_to_matrix_kernel(const double* __restrict__ probe, int K, int out_rows, int rows, int Kpad,
                                       double diag, const double* __restrict__ coef, int P1,
                                       const int4* __restrict__ modes, float* __restrict__ hi,
                                       float* __restrict__ lo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * Kpad) return;
    const int r = (int)(i / Kpad), k = (int)(i - (long long)r * Kpad);
    double v = 0.0;
    if (k < K) {
        if (r < out_rows) {
            v = probe[(long long)k * K + r] + (r == k ? diag : 0.0);
        } else {
            const int4 md = modes[r - out_rows];  // type, n, m, part
            const double* cg = coef + (long long)k * 3 * P1 * P1 * 2;
            v = cg[2 * (md.x * P1 * P1 + md.y * P1 + md.z) + md.w];
        }
    }
    const float h = tf32_hi((float)v);
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
}

__global__ void unit_columns_kernel(int K, double* __restrict__ d) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)K * K) return;
    d[i] = (i / K == i % K) ? 1.0 : 0.0;
}

__global__ void to_float_kernel(int n, const double* __restrict__ x, float* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

__global__ void fill_kernel(long long n, double v, double* __restrict__ d) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = v;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// 2-D FP32 tensor [rows][Kpad] read as boxes of box_rows x 32 with the
// 128-byte swizzle; columns K..Kpad-1 and rows past `rows` read as zero.
bool make_map(CUtensorMap* m, float* base, int rows, int K, int Kpad, int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kpad * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Device state of the self-term GEMMs of one context (one VSH order).
struct SelfGemm {
    int K = 0, Kpad = 0;
    int rows[kSelfMats] = {0, 0, 0};
    float* mat[kSelfMats] = {nullptr, nullptr, nullptr};  // hi [rows][Kpad] followed by lo
    CUtensorMap mh[kSelfMats], ml[kSelfMats];
    float* b = nullptr;  // density operand: hi [n][Kpad] followed by lo
    float* af = nullptr; // [n] radii in FP32 (the single layer's scale)
    CUtensorMap bh, bl;
    int* err = nullptr;
};

void self_gemm_free(sbie_ctx* c) {
    if (!c->sg) return;
    for (int i = 0; i < kSelfMats; ++i) cudaFree(c->sg->mat[i]);
    cudaFree(c->sg->b);
    cudaFree(c->sg->af);
    cudaFree(c->sg->err);
    delete c->sg;
    c->sg = nullptr;
}

bool self_gemm_ready(const sbie_ctx* c, int which) { return c->sg && c->sg->mat[which]; }

cudaError_t self_gemm_build(sbie_ctx* c, int which) {
    if (self_gemm_ready(c, which)) return cudaSuccess;
    if (!encode_fn()) return cudaErrorNotSupported;
    cudaError_t e = cudaSuccess;
    if (!c->sg) {
        SelfGemm* g = new SelfGemm;
        g->K = 3 * c->npn;
        g->Kpad = (g->K + kBK - 1) / kBK * kBK;
        const size_t nb = (size_t)c->n * g->Kpad;
        e = cudaMalloc(&g->b, sizeof(float) * 2 * nb);
        if (e == cudaSuccess) e = cudaMalloc(&g->af, sizeof(float) * c->n);
        if (e == cudaSuccess) {
            to_float_kernel<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, c->d_a, g->af);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMalloc(&g->err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(g->err, 0, sizeof(int), c->stream);
        if (e == cudaSuccess && (!make_map(&g->bh, g->b, c->n, g->K, g->Kpad, kBN) ||
                                 !make_map(&g->bl, g->b + nb, c->n, g->K, g->Kpad, kBN)))
            e = cudaErrorInvalidValue;
        if (e != cudaSuccess) {
            cudaFree(g->b);
            cudaFree(g->af);
            cudaFree(g->err);
            delete g;
            return e;
        }
        c->sg = g;
    }
    SelfGemm* g = c->sg;
    const int K = g->K, Kpad = g->Kpad, P1 = c->p + 1;
    const bool prec = which == kSelfPrec;
    const int rows = K + (prec ? kLowModes : 0);
    // probe: the FP64 self kernel on K unit densities (unit radius), and for
    // the preconditioner the coefficients of each probe column
    double *dens = nullptr, *out = nullptr, *one = nullptr, *coef = nullptr;
    float* mat = nullptr;
    const size_t KK = (size_t)K * K;
    e = cudaMalloc(&dens, sizeof(double) * KK);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * KK);
    if (e == cudaSuccess) e = cudaMalloc(&one, sizeof(double) * K);
    if (e == cudaSuccess && prec) e = cudaMalloc(&coef, sizeof(double) * (size_t)K * 3 * P1 * P1 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&mat, sizeof(float) * 2 * (size_t)rows * Kpad);
    if (e == cudaSuccess) {
        unit_columns_kernel<<<(unsigned)((KK + 255) / 256), 256, 0, c->stream>>>(K, dens);
        fill_kernel<<<(K + 255) / 256, 256, 0, c->stream>>>(K, 1.0, one);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int op = which == kSelfS ? (int)Kern::S : (which == kSelfDK ? (int)Kern::D : kOpPrecHigh);
        e = launch_self_probe(c, op, K, dens, out, one, coef);
    }
    if (e == cudaSuccess) {
        const long long tot = (long long)rows * Kpad;
        probe_to_matrix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(
            out, K, K, rows, Kpad, prec ? 2.0 : 0.0, coef, P1, c->d_modes, mat, mat + (size_t)rows * Kpad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dens);
    cudaFree(out);
    cudaFree(one);
    cudaFree(coef);
    if (e == cudaSuccess && (!make_map(&g->mh[which], mat, rows, K, Kpad, kBM) ||
                             !make_map(&g->ml[which], mat + (size_t)rows * Kpad, rows, K, Kpad, kBM)))
        e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        cudaFree(mat);
        return e;
    }
    g->mat[which] = mat;
    g->rows[which] = rows;
    return cudaSuccess;
}

cudaError_t launch_self_gemm(sbie_ctx* c, int which, const double* dens, double* out, bool accumulate) {
    SelfGemm* g = c->sg;
    if (!g || !g->mat[which]) return cudaErrorInvalidValue;
    const size_t nb = (size_t)c->n * g->Kpad;
    {
        const long long tot = (long long)c->n * g->Kpad;
        split_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(dens, g->K, c->n, g->K, g->Kpad,
                                                                                 g->b, g->b + nb);
        ++c->n_launch;
    }
    GemmEpi E;
    E.rows = g->rows[which];
    E.out_rows = g->K;
    E.cols = c->n;
    E.ld_out = g->K;
    E.out = out;
    E.accumulate = accumulate ? 1 : 0;
    E.scale = which == kSelfS ? g->af : nullptr;
    E.low = which == kSelfPrec ? c->d_low : nullptr;
    E.k_blocks = g->Kpad / kBK;
    E.k_total = E.k_blocks;
    E.exact = 0;
    E.err = g->err;
    cudaError_t e =
        cudaFuncSetAttribute(self_gemm_kernel<GemmEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 grid((E.rows + kBM - 1) / kBM, (c->n + kBN - 1) / kBN);
    self_gemm_kernel<GemmEpi><<<grid, 128, kSmemBytes, c->stream>>>(g->mh[which], g->ml[which], g->bh, g->bl, E);
    ++c->n_launch;
    return cudaGetLastError();
}

// Split-K reduction of tc_gemm_tf32: C[n ldc + m] = epilogue(sum_z part[z][n][m]).
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ part, TcEpi ep) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * N) return;
    const int n = (int)(i / M), m = (int)(i - (long long)n * M);
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += part[(long long)z * M * N + i];
    if (ep.mode == TcEpi::kBias || ep.mode == TcEpi::kBiasTanh) v += ep.bias[m];
    if (ep.mode == TcEpi::kBiasTanh) v = tanhf(v);
    if (ep.mode == TcEpi::kDTanh) {
        const float g = ep.G[(long long)n * ep.ldg + m];
        v *= 1.f - g * g;
    }
    ep.C[(long long)n * ep.ldc + m] = v;
}

// (A B^T)^T (+ epilogue) for the pair network: A [M][Kpad] and B [N][Kpad] as
// TF32 high parts and remainders (zero past K); a null remainder marks an
// operand exact in TF32 (the BF16 weights), whose remainder products are
// skipped.  Output (m, n) goes to C[n ldc + m].  A long K over few output tiles is
// split over up to `work_cap / (M N)` slices of at least 4 K blocks each,
// whose raw sums `work` holds until one reduction kernel adds them in a fixed
// order and applies the epilogue.
cudaError_t tc_gemm_tf32(cudaStream_t s, int M, int N, int Kpad, const float* Ahi, const float* Alo,
                         const float* Bhi, const float* Blo, const TcEpi& ep, int* err, float* work,
                         size_t work_cap) {
    if (M <= 0 || N <= 0 || Kpad <= 0 || Kpad % kBK || (!Alo && !Blo)) return cudaErrorInvalidValue;
    if (!encode_fn()) return cudaErrorNotSupported;
    CUtensorMap ah, al, bh, bl;
    if (!make_map(&ah, const_cast<float*>(Ahi), M, Kpad, Kpad, kBM) ||
        !make_map(&al, const_cast<float*>(Alo ? Alo : Ahi), M, Kpad, Kpad, kBM) ||
        !make_map(&bh, const_cast<float*>(Bhi), N, Kpad, Kpad, kBN) ||
        !make_map(&bl, const_cast<float*>(Blo ? Blo : Bhi), N, Kpad, Kpad, kBN))
        return cudaErrorInvalidValue;
    const int kblocks = Kpad / kBK, tiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
    int splits = 1;
    if (work && tiles < 76) {
        splits = std::min(kblocks / 4, (152 + tiles - 1) / tiles);
        splits = (int)std::min<long long>(splits, (long long)(work_cap / ((size_t)M * N)));
        splits = std::max(splits, 1);
    }
    const int per = (kblocks + splits - 1) / splits;
    splits = (kblocks + per - 1) / per;  // no empty slice
    MlpEpi E;
    E.M = M;
    E.N = N;
    E.ldc = splits > 1 ? M : ep.ldc;
    E.ldg = ep.ldg;
    E.C = splits > 1 ? work : ep.C;
    E.bias = ep.bias;
    E.G = ep.G;
    E.mode = splits > 1 ? TcEpi::kNone : ep.mode;
    E.k_blocks = per;
    E.k_total = kblocks;
    E.exact = (Alo ? 0 : 1) | (Blo ? 0 : 2);
    E.err = err;
    E.zstride = (long long)M * N;
    // (under stream capture the attribute was set by an earlier eager call on this device)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e == cudaSuccess && cap == cudaStreamCaptureStatusNone)
        e = cudaFuncSetAttribute(self_gemm_kernel<MlpEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 grid((M + kBM - 1) / kBM, (N + kBN - 1) / kBN, splits);
    self_gemm_kernel<MlpEpi><<<grid, 128, kSmemBytes, s>>>(ah, al, bh, bl, E);
    if ((e = cudaGetLastError()) != cudaSuccess || splits == 1) return e;
    const long long tot = (long long)M * N;
    splitk_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, N, splits, work, ep);
    return cudaGetLastError();
}

cudaError_t self_gemm_error(sbie_ctx* c, int* flag) {
    *flag = 0;
    if (!c->sg) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(flag, c->sg->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e;
}

}  // namespace sbie
