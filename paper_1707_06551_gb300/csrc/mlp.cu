// The pair network of the learned preconditioner: a fully connected
// 5 -> 128 -> 128 -> 128 -> 73*73 network with tanh activations that maps the
// geometry of a close pair (target offset in the pair frame, source radius,
// target radius; standardised) to its standardised low-mode interaction block.
// Weights are kept in FP32 (Adam) and used in BF16 by the forward and backward
// passes, which accumulate in FP32.  Hand-written kernels: one tiled GEMM
// template (both operands row-major, either transposed, float or BF16) with
// fused bias / tanh / tanh-derivative epilogues, column sums, the loss and
// Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "common.h"
#include "mlp.h"

namespace sbie {

namespace {

template <typename T>
__device__ __forceinline__ float ld(const T* p) {
    return (float)(*p);
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}

enum Epi { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_TANH = 2, EPI_DTANH = 3 };

// C[M][N] = sum_k A(m, k) B(k, n) (+ epilogue).  A(m, k) = TA ? A[k lda + m]
// : A[m lda + k]; B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  64 x 64 tiles,
// 256 threads, 4 x 4 outputs per thread, K step 16.  EPI_DTANH multiplies by
// (1 - G[m][n]^2) (the tanh derivative of the layer's output G).
template <typename TA_, typename TB_, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const TA_* __restrict__ A, int lda,
                                                   const TB_* __restrict__ B, int ldb, const float* __restrict__ bias,
                                                   const float* __restrict__ G, float* __restrict__ C) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            int kk = e / 64, mm = e % 64;
            int m = m0 + mm, k = k0 + kk;
            float va = 0.f;
            if (m < M && k < K) va = TA ? ld(A + (size_t)k * lda + m) : ld(A + (size_t)m * lda + k);
            As[kk][mm] = va;
            int n = n0 + mm;
            float vb = 0.f;
            if (n < N && k < K) vb = TB ? ld(B + (size_t)n * ldb + k) : ld(B + (size_t)k * ldb + n);
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (EPI == EPI_BIAS || EPI == EPI_BIAS_TANH) v += bias[n];
            if (EPI == EPI_BIAS_TANH) v = tanhf(v);
            if (EPI == EPI_DTANH) {
                float g = G[(size_t)m * N + n];
                v *= 1.f - g * g;
            }
            C[(size_t)m * N + n] = v;
        }
    }
}

template <typename TA_, typename TB_, bool TA, bool TB, int EPI>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const TA_* A, int lda, const TB_* B, int ldb, const float* bias,
                 const float* G, float* C) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<TA_, TB_, TA, TB, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, G, C);
    return cudaGetLastError();
}

// out[n] = sum_m D[m][n]
__global__ void colsum_kernel(int M, int N, const float* __restrict__ D, float* __restrict__ out) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += D[(size_t)m * N + n];
    out[n] = s;
}

// dY = 2 (Y - T) / (M N); partial sums of the squared error per block
__global__ void loss_kernel(long long total, float scale, const float* __restrict__ Y, const float* __restrict__ T,
                            float* __restrict__ dY, double* __restrict__ partial) {
    __shared__ double sh[256];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        float d = Y[i] - T[i];
        s += (double)d * d;
        if (dY) dY[i] = 2.f * d * scale;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void adam_kernel(long long n, float lr, float b1, float b2, float eps, float c1, float c2,
                            float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, __nv_bfloat16* __restrict__ wb) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float a = b1 * m1[i] + (1.f - b1) * gi;
    float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float v = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[i] = v;
    wb[i] = __float2bfloat16(v);
}

__global__ void to_bf16_kernel(long long n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16(w[i]);
}

__global__ void gather_rows_kernel(int n, int width, const int* __restrict__ idx, const float* __restrict__ src,
                                   float* __restrict__ dst) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * width) return;
    int r = (int)(e / width), c = (int)(e - (long long)r * width);
    dst[e] = src[(size_t)idx[r] * width + c];
}

}  // namespace

MlpLayout mlp_layout() {
    MlpLayout L{};
    const int in[4] = {kMlpIn, kMlpHidden, kMlpHidden, kMlpHidden};
    const int out[4] = {kMlpHidden, kMlpHidden, kMlpHidden, kMlpOut};
    long long o = 0;
    for (int l = 0; l < 4; ++l) {
        L.din[l] = in[l];
        L.dout[l] = out[l];
        L.w[l] = o;
        o += (long long)in[l] * out[l];
        L.b[l] = o;
        o += out[l];
    }
    L.total = o;
    return L;
}

// Device workspace for a batch of up to `cap` rows.
struct MlpWork {
    int cap = 0;
    float* h[4] = {nullptr, nullptr, nullptr, nullptr};  // layer outputs (h[3] = network output)
    float* d[4] = {nullptr, nullptr, nullptr, nullptr};  // gradients w.r.t. layer outputs
    double* partial = nullptr;
    cudaError_t alloc(int c) {
        cap = c;
        MlpLayout L = mlp_layout();
        for (int l = 0; l < 4; ++l) {
            if (cudaMalloc(&h[l], sizeof(float) * (size_t)c * L.dout[l]) != cudaSuccess) return cudaErrorMemoryAllocation;
            if (cudaMalloc(&d[l], sizeof(float) * (size_t)c * L.dout[l]) != cudaSuccess) return cudaErrorMemoryAllocation;
        }
        return cudaMalloc(&partial, sizeof(double) * 1024);
    }
    void release() {
        for (int l = 0; l < 4; ++l) {
            if (h[l]) cudaFree(h[l]);
            if (d[l]) cudaFree(d[l]);
            h[l] = d[l] = nullptr;
        }
        if (partial) cudaFree(partial);
        partial = nullptr;
    }
};

// Forward pass of B rows X [B][5] with BF16 weights wb (FP32 biases from w).
static cudaError_t forward(cudaStream_t s, const MlpLayout& L, const float* w, const __nv_bfloat16* wb, int B,
                           const float* X, MlpWork& ws) {
    cudaError_t e = gemm<float, __nv_bfloat16, false, false, EPI_BIAS_TANH>(s, B, L.dout[0], L.din[0], X, L.din[0],
                                                                            wb + L.w[0], L.dout[0], w + L.b[0], nullptr,
                                                                            ws.h[0]);
    for (int l = 1; l < 3 && e == cudaSuccess; ++l)
        e = gemm<float, __nv_bfloat16, false, false, EPI_BIAS_TANH>(s, B, L.dout[l], L.din[l], ws.h[l - 1], L.din[l],
                                                                    wb + L.w[l], L.dout[l], w + L.b[l], nullptr, ws.h[l]);
    if (e == cudaSuccess)
        e = gemm<float, __nv_bfloat16, false, false, EPI_BIAS>(s, B, L.dout[3], L.din[3], ws.h[2], L.din[3], wb + L.w[3],
                                                               L.dout[3], w + L.b[3], nullptr, ws.h[3]);
    return e;
}

// Loss (mean squared error over the B x out entries) and its gradient `grad`
// (FP32, same layout as w).  *loss_dev receives the block partial sums.
static cudaError_t backward(cudaStream_t s, const MlpLayout& L, const __nv_bfloat16* wb, int B, const float* X,
                            const float* T, MlpWork& ws, float* grad, int* nblk) {
    const long long total = (long long)B * L.dout[3];
    const int blocks = (int)std::min<long long>(1024, (total + 255) / 256);
    *nblk = blocks;
    loss_kernel<<<blocks, 256, 0, s>>>(total, 1.f / (float)total, ws.h[3], T, ws.d[3], ws.partial);
    cudaError_t e = cudaGetLastError();
    for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
        const float* Ain = l == 0 ? X : ws.h[l - 1];
        // dW_l = A_in^T dZ_l ; db_l = colsum(dZ_l)
        e = gemm<float, float, true, false, EPI_NONE>(s, L.din[l], L.dout[l], B, Ain, L.din[l], ws.d[l], L.dout[l],
                                                      nullptr, nullptr, grad + L.w[l]);
        if (e != cudaSuccess) break;
        colsum_kernel<<<(L.dout[l] + 255) / 256, 256, 0, s>>>(B, L.dout[l], ws.d[l], grad + L.b[l]);
        e = cudaGetLastError();
        if (l == 0 || e != cudaSuccess) break;
        // dZ_{l-1} = (dZ_l W_l^T) (1 - h_{l-1}^2)
        e = gemm<float, __nv_bfloat16, false, true, EPI_DTANH>(s, B, L.din[l], L.dout[l], ws.d[l], L.dout[l],
                                                               wb + L.w[l], L.dout[l], nullptr, ws.h[l - 1], ws.d[l - 1]);
    }
    return e;
}

static double read_loss(cudaStream_t s, const MlpWork& ws, int nblk, long long total, cudaError_t* err) {
    double part[1024];
    *err = cudaMemcpyAsync(part, ws.partial, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(s);
    double t = 0.0;
    for (int i = 0; i < nblk; ++i) t += part[i];
    return t / (double)total;
}

cudaError_t mlp_gradients(const float* h_params, int n, const float* h_X, const float* h_T, float* h_grad,
                          double* loss) {
    MlpLayout L = mlp_layout();
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    float *w = nullptr, *g = nullptr, *X = nullptr, *T = nullptr;
    __nv_bfloat16* wb = nullptr;
    MlpWork ws;
    int nblk = 0;
    e = cudaMalloc(&w, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&g, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&wb, sizeof(__nv_bfloat16) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&X, sizeof(float) * (size_t)n * kMlpIn);
    if (e == cudaSuccess) e = cudaMalloc(&T, sizeof(float) * (size_t)n * kMlpOut);
    if (e == cudaSuccess) e = ws.alloc(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, h_params, sizeof(float) * L.total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, h_X, sizeof(float) * (size_t)n * kMlpIn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T, h_T, sizeof(float) * (size_t)n * kMlpOut, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        to_bf16_kernel<<<(unsigned)((L.total + 255) / 256), 256, 0, s>>>(L.total, w, wb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = forward(s, L, w, wb, n, X, ws);
    if (e == cudaSuccess) e = backward(s, L, wb, n, X, T, ws, g, &nblk);
    if (e == cudaSuccess) *loss = read_loss(s, ws, nblk, (long long)n * kMlpOut, &e);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_grad, g, sizeof(float) * L.total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ws.release();
    for (void* p : {(void*)w, (void*)g, (void*)wb, (void*)X, (void*)T})
        if (p) cudaFree(p);
    cudaStreamDestroy(s);
    return e;
}

cudaError_t mlp_forward_dev(cudaStream_t s, const float* w, const __nv_bfloat16* wb, int n, const float* X, float* Y) {
    MlpLayout L = mlp_layout();
    MlpWork ws;
    const int chunk = 4096;
    cudaError_t e = ws.alloc(std::min(n, chunk));
    for (int r = 0; r < n && e == cudaSuccess; r += chunk) {
        int b = std::min(chunk, n - r);
        e = forward(s, L, w, wb, b, X + (size_t)r * kMlpIn, ws);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Y + (size_t)r * kMlpOut, ws.h[3], sizeof(float) * (size_t)b * kMlpOut,
                                cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ws.release();
    return e;
}

cudaError_t mlp_to_bf16(cudaStream_t s, const float* w, __nv_bfloat16* wb) {
    MlpLayout L = mlp_layout();
    to_bf16_kernel<<<(unsigned)((L.total + 255) / 256), 256, 0, s>>>(L.total, w, wb);
    return cudaGetLastError();
}

// Adam training on standardised data X [n][5], T [n][out] (host, FP32).
cudaError_t mlp_train(const MlpTrainOpts& o, int n, const float* h_X, const float* h_T, float* h_params,
                      std::vector<double>& history) {
    MlpLayout L = mlp_layout();
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr, *X = nullptr, *T = nullptr, *Xb = nullptr,
          *Tb = nullptr;
    int* idx = nullptr;
    __nv_bfloat16* wb = nullptr;
    MlpWork ws;
    const int B = std::max(1, std::min(o.batch, n));
    e = cudaMalloc(&w, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&g, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&m1, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&m2, sizeof(float) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&wb, sizeof(__nv_bfloat16) * L.total);
    if (e == cudaSuccess) e = cudaMalloc(&X, sizeof(float) * (size_t)n * kMlpIn);
    if (e == cudaSuccess) e = cudaMalloc(&T, sizeof(float) * (size_t)n * kMlpOut);
    if (e == cudaSuccess) e = cudaMalloc(&Xb, sizeof(float) * (size_t)B * kMlpIn);
    if (e == cudaSuccess) e = cudaMalloc(&Tb, sizeof(float) * (size_t)B * kMlpOut);
    if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = ws.alloc(B);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, h_params, sizeof(float) * L.total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m1, 0, sizeof(float) * L.total, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m2, 0, sizeof(float) * L.total, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, h_X, sizeof(float) * (size_t)n * kMlpIn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T, h_T, sizeof(float) * (size_t)n * kMlpOut, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = mlp_to_bf16(s, w, wb);
    std::mt19937_64 rng(o.seed);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    long long step = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < o.epochs && e == cudaSuccess; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        e = cudaMemcpyAsync(idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
        double ep_loss = 0.0;
        int nb_steps = 0;
        for (int r = 0; r + B <= n && e == cudaSuccess; r += B) {
            gather_rows_kernel<<<(B * kMlpIn + 255) / 256, 256, 0, s>>>(B, kMlpIn, idx + r, X, Xb);
            gather_rows_kernel<<<(unsigned)(((long long)B * kMlpOut + 255) / 256), 256, 0, s>>>(B, kMlpOut, idx + r, T, Tb);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = forward(s, L, w, wb, B, Xb, ws);
            int nblk = 0;
            if (e == cudaSuccess) e = backward(s, L, wb, B, Xb, Tb, ws, g, &nblk);
            ++step;
            const float lr = (float)(o.lr * (ep < o.epochs / 2 ? 1.0 : (ep < 3 * o.epochs / 4 ? 0.3 : 0.1)));
            if (e == cudaSuccess) {
                adam_kernel<<<(unsigned)((L.total + 255) / 256), 256, 0, s>>>(
                    L.total, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step), w, g, m1, m2, wb);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess && r + 2 * B > n) ep_loss = read_loss(s, ws, nblk, (long long)B * kMlpOut, &e);
            ++nb_steps;
        }
        history.push_back(ep_loss);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_params, w, sizeof(float) * L.total, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ws.release();
    for (void* p : {(void*)w, (void*)g, (void*)m1, (void*)m2, (void*)wb, (void*)X, (void*)T, (void*)Xb, (void*)Tb,
                    (void*)idx})
        if (p) cudaFree(p);
    cudaStreamDestroy(s);
    return e;
}

void mlp_init(unsigned long long seed, std::vector<float>& params) {
    MlpLayout L = mlp_layout();
    params.assign(L.total, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 4; ++l) {
        std::normal_distribution<float> nd(0.f, 1.f / std::sqrt((float)L.din[l]));
        for (long long i = 0; i < (long long)L.din[l] * L.dout[l]; ++i) params[L.w[l] + i] = nd(rng);
    }
}

}  // namespace sbie
