// The pair network of the learned preconditioner: a fully connected
// 5 -> 128 -> 128 -> 128 -> 73*73 network with tanh activations that maps the
// geometry of a close pair (target offset in the pair frame, source radius,
// target radius; standardised) to its standardised low-mode interaction block.
// Weights are kept in FP32 (Adam) and used in BF16 by the forward and backward
// passes, which accumulate in FP32.  Every layer's GEMM (forward, weight
// gradient, input gradient) runs on the tensor cores (tc_gemm_tf32 of
// selfgemm.cu: tcgen05, 3xTF32 -- the BF16 weights are exact in TF32, the FP32
// activations and gradients are split into TF32 high parts and remainders),
// with the bias / tanh / tanh-derivative epilogues fused.  Here: the operand
// packing (K-major TF32 pairs, zero-padded, transposed where the product needs
// it), column sums, the loss and Adam.
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

// Operand packing for tc_gemm_tf32: dst [rows][Kpad] (TF32 high part, and the
// remainder when lo is given), dst[r][k] = src[r lds + k] for k < K, zero for
// K <= k < Kpad.
template <typename T>
__global__ void pack_kernel(const T* __restrict__ src, long long lds, int rows, int K, int Kpad,
                            float* __restrict__ hi, float* __restrict__ lo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * Kpad) return;
    const long long r = i / Kpad;
    const int k = (int)(i - r * Kpad);
    const float v = k < K ? ld(src + r * lds + k) : 0.f;
    const float h = tf32_hi(v);
    hi[i] = h;
    if (lo) lo[i] = v - h;
}

// Transposed packing through 32 x 32 shared-memory tiles: dst[r][k] =
// src[k lds + r] for r < rows, k < K (src has K rows of at least `rows` values).
template <typename T>
__global__ void pack_t_kernel(const T* __restrict__ src, long long lds, int rows, int K, int Kpad,
                              float* __restrict__ hi, float* __restrict__ lo) {
    __shared__ float tile[32][33];
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int j = ty; j < 32; j += 8) {
        const int k = k0 + j, r = r0 + tx;
        tile[j][tx] = (k < K && r < rows) ? ld(src + (long long)k * lds + r) : 0.f;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int r = r0 + j, k = k0 + tx;
        if (r >= rows || k >= Kpad) continue;
        const float v = tile[tx][j];
        const float h = tf32_hi(v);
        hi[(long long)r * Kpad + k] = h;
        if (lo) lo[(long long)r * Kpad + k] = v - h;
    }
}

inline int pad32(int k) { return (k + 31) / 32 * 32; }

template <typename T>
cudaError_t pack(cudaStream_t s, const T* src, long long ld, int rows, int K, int Kpad, float* hi, float* lo) {
    const long long tot = (long long)rows * Kpad;
    pack_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, ld, rows, K, Kpad, hi, lo);
    return cudaGetLastError();
}
template <typename T>
cudaError_t pack_t(cudaStream_t s, const T* src, long long ld, int rows, int K, int Kpad, float* hi, float* lo) {
    dim3 grid((rows + 31) / 32, (Kpad + 31) / 32);
    pack_t_kernel<T><<<grid, 256, 0, s>>>(src, ld, rows, K, Kpad, hi, lo);
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

// Adam with its step size and bias corrections read from the device
// (hyper[0] = learning rate, hyper[1] = 1 - b1^t, hyper[2] = 1 - b2^t), so
// that one captured epoch replays every epoch.
__global__ void adam_kernel(long long n, const float* __restrict__ hyper, float b1, float b2, float eps,
                            float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, __nv_bfloat16* __restrict__ wb) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float lr = hyper[0], c1 = hyper[1], c2 = hyper[2];
    float gi = g[i];
    float a = b1 * m1[i] + (1.f - b1) * gi;
    float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float v = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[i] = v;
    wb[i] = __float2bfloat16(v);
}

// t <- t + 1 and the bias corrections of step t
__global__ void adam_step_kernel(int* __restrict__ t, float* __restrict__ hyper, float b1, float b2) {
    const int s = ++*t;
    hyper[1] = 1.f - powf(b1, (float)s);
    hyper[2] = 1.f - powf(b2, (float)s);
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

// Device workspace for a batch of up to `cap` rows; `train` adds the
// gradients and the operand space of the backward GEMMs.
struct MlpWork {
    int cap = 0;
    float* h[4] = {nullptr, nullptr, nullptr, nullptr};  // layer outputs (h[3] = network output)
    float* d[4] = {nullptr, nullptr, nullptr, nullptr};  // gradients w.r.t. layer outputs
    double* partial = nullptr;
    float* pa = nullptr;  // A operand: high parts, then remainders
    float* pb = nullptr;  // B operand: high parts, then remainders
    size_t na = 0, nb = 0;
    float* work = nullptr;  // split-K partial sums of the input-gradient GEMMs
    size_t nwork = 0;
    int* err = nullptr;   // bounded-wait flag of the tensor-core GEMMs
    cudaError_t alloc(int c, bool train) {
        cap = c;
        MlpLayout L = mlp_layout();
        for (int l = 0; l < 4; ++l) {
            if (cudaMalloc(&h[l], sizeof(float) * (size_t)c * L.dout[l]) != cudaSuccess) return cudaErrorMemoryAllocation;
            if (train && cudaMalloc(&d[l], sizeof(float) * (size_t)c * L.dout[l]) != cudaSuccess)
                return cudaErrorMemoryAllocation;
        }
        // forward: A = layer input [c][din], B = W^T [dout][din]; backward:
        // A = dZ [c][dout] or input^T [din][c], B = W [din][dout] or dZ^T [dout][c]
        for (int l = 0; l < 4; ++l) {
            na = std::max(na, (size_t)c * pad32(L.din[l]));
            nb = std::max(nb, (size_t)L.dout[l] * pad32(L.din[l]));
            if (train) {
                na = std::max(na, std::max((size_t)c * pad32(L.dout[l]), (size_t)L.din[l] * pad32(c)));
                nb = std::max(nb, std::max((size_t)L.din[l] * pad32(L.dout[l]), (size_t)L.dout[l] * pad32(c)));
            }
        }
        if (cudaMalloc(&pa, sizeof(float) * 2 * na) != cudaSuccess) return cudaErrorMemoryAllocation;
        if (cudaMalloc(&pb, sizeof(float) * 2 * nb) != cudaSuccess) return cudaErrorMemoryAllocation;
        if (train) {  // up to 32 slices of the largest input gradient [c][din]
            nwork = (size_t)32 * c * kMlpHidden;
            if (cudaMalloc(&work, sizeof(float) * nwork) != cudaSuccess) return cudaErrorMemoryAllocation;
        }
        if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return cudaErrorMemoryAllocation;
        if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess) return cudaErrorMemoryAllocation;
        return cudaMalloc(&partial, sizeof(double) * 1024);
    }
    // cudaErrorLaunchTimeout when a GEMM's bounded wait ran out
    cudaError_t check(cudaStream_t s) const {
        int flag = 0;
        cudaError_t e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && flag) e = cudaErrorLaunchTimeout;
        return e;
    }
    void release() {
        for (int l = 0; l < 4; ++l) {
            if (h[l]) cudaFree(h[l]);
            if (d[l]) cudaFree(d[l]);
            h[l] = d[l] = nullptr;
        }
        for (void* p : {(void*)partial, (void*)pa, (void*)pb, (void*)err, (void*)work})
            if (p) cudaFree(p);
        partial = nullptr;
        pa = pb = work = nullptr;
        err = nullptr;
    }
};

// Forward pass of B rows X [B][5] with BF16 weights wb (FP32 biases from w):
// h_l = tanh(h_{l-1} W_l + b_l), the last layer without tanh.
static cudaError_t forward(cudaStream_t s, const MlpLayout& L, const float* w, const __nv_bfloat16* wb, int B,
                           const float* X, MlpWork& ws) {
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        const int din = L.din[l], dout = L.dout[l], Kp = pad32(din);
        e = pack(s, l == 0 ? X : ws.h[l - 1], din, B, din, Kp, ws.pa, ws.pa + ws.na);
        if (e == cudaSuccess) e = pack_t(s, wb + L.w[l], dout, dout, din, Kp, ws.pb, (float*)nullptr);
        TcEpi ep;
        ep.C = ws.h[l];
        ep.ldc = dout;
        ep.bias = w + L.b[l];
        ep.mode = l < 3 ? TcEpi::kBiasTanh : TcEpi::kBias;
        // (W^T H^T)^T: the output features on the TMEM lanes (coalesced stores)
        if (e == cudaSuccess) e = tc_gemm_tf32(s, dout, B, Kp, ws.pb, nullptr, ws.pa, ws.pa + ws.na, ep, ws.err);
    }
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
    const int Kb = pad32(B);
    for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
        const float* Ain = l == 0 ? X : ws.h[l - 1];
        const int din = L.din[l], dout = L.dout[l];
        // dW_l = A_in^T dZ_l = ((dZ_l^T) (A_in^T)^T)^T  (GEMM M = dout, N = din, K = B)
        e = pack_t(s, Ain, din, din, B, Kb, ws.pa, ws.pa + ws.na);
        if (e == cudaSuccess) e = pack_t(s, ws.d[l], dout, dout, B, Kb, ws.pb, ws.pb + ws.nb);
        TcEpi gw;
        gw.C = grad + L.w[l];
        gw.ldc = dout;
        if (e == cudaSuccess) e = tc_gemm_tf32(s, dout, din, Kb, ws.pb, ws.pb + ws.nb, ws.pa, ws.pa + ws.na, gw, ws.err);
        if (e != cudaSuccess) break;
        // db_l = colsum(dZ_l)
        colsum_kernel<<<(dout + 255) / 256, 256, 0, s>>>(B, dout, ws.d[l], grad + L.b[l]);
        e = cudaGetLastError();
        if (l == 0 || e != cudaSuccess) break;
        // dZ_{l-1} = (dZ_l W_l^T) (1 - h_{l-1}^2) = (W_l dZ_l^T)^T ...  (GEMM M = din, N = B, K = dout)
        const int Kd = pad32(dout);
        e = pack(s, ws.d[l], dout, B, dout, Kd, ws.pa, ws.pa + ws.na);
        if (e == cudaSuccess) e = pack(s, wb + L.w[l], dout, din, dout, Kd, ws.pb, (float*)nullptr);
        TcEpi gz;
        gz.C = ws.d[l - 1];
        gz.ldc = din;
        gz.G = ws.h[l - 1];
        gz.ldg = din;
        gz.mode = TcEpi::kDTanh;
        if (e == cudaSuccess)
            e = tc_gemm_tf32(s, din, B, Kd, ws.pb, nullptr, ws.pa, ws.pa + ws.na, gz, ws.err, ws.work, ws.nwork);
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
    if (e == cudaSuccess) e = ws.alloc(n, true);
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
    if (e == cudaSuccess) e = ws.check(s);
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
    cudaError_t e = ws.alloc(std::min(n, chunk), false);
    for (int r = 0; r < n && e == cudaSuccess; r += chunk) {
        int b = std::min(chunk, n - r);
        e = forward(s, L, w, wb, b, X + (size_t)r * kMlpIn, ws);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(Y + (size_t)r * kMlpOut, ws.h[3], sizeof(float) * (size_t)b * kMlpOut,
                                cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = ws.check(s);
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
    if (e == cudaSuccess) e = ws.alloc(B, true);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w, h_params, sizeof(float) * L.total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m1, 0, sizeof(float) * L.total, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m2, 0, sizeof(float) * L.total, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, h_X, sizeof(float) * (size_t)n * kMlpIn, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T, h_T, sizeof(float) * (size_t)n * kMlpOut, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = mlp_to_bf16(s, w, wb);
    float* hyper = nullptr;  // learning rate, bias corrections
    int* tstep = nullptr;    // Adam step counter
    if (e == cudaSuccess) e = cudaMalloc(&hyper, sizeof(float) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&tstep, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(tstep, 0, sizeof(int), s);
    std::mt19937_64 rng(o.seed);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    const float b1 = 0.9f, b2 = 0.999f;
    int nblk = 0;
    // one epoch: every mini-batch of the shuffled order in idx
    auto epoch = [&]() -> cudaError_t {
        cudaError_t er = cudaSuccess;
        for (int r = 0; r + B <= n && er == cudaSuccess; r += B) {
            gather_rows_kernel<<<(B * kMlpIn + 255) / 256, 256, 0, s>>>(B, kMlpIn, idx + r, X, Xb);
            gather_rows_kernel<<<(unsigned)(((long long)B * kMlpOut + 255) / 256), 256, 0, s>>>(B, kMlpOut, idx + r, T,
                                                                                               Tb);
            er = cudaGetLastError();
            if (er == cudaSuccess) er = forward(s, L, w, wb, B, Xb, ws);
            if (er == cudaSuccess) er = backward(s, L, wb, B, Xb, Tb, ws, g, &nblk);
            if (er == cudaSuccess) {
                adam_step_kernel<<<1, 1, 0, s>>>(tstep, hyper, b1, b2);
                adam_kernel<<<(unsigned)((L.total + 255) / 256), 256, 0, s>>>(L.total, hyper, b1, b2, 1e-8f, w, g, m1,
                                                                               m2, wb);
                er = cudaGetLastError();
            }
        }
        return er;
    };
    // The first epoch runs launch by launch; the second is captured as a CUDA
    // graph, which every later epoch replays (the shuffled order and the
    // learning rate are copied to the device before each epoch).
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    for (int ep = 0; ep < o.epochs && e == cudaSuccess; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        const float lr = (float)(o.lr * (ep < o.epochs / 2 ? 1.0 : (ep < 3 * o.epochs / 4 ? 0.3 : 0.1)));
        e = cudaMemcpyAsync(idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hyper, &lr, sizeof(float), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && ep == 0) {
            e = epoch();
        } else if (e == cudaSuccess) {
            if (!exec) {
                e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t ec = epoch();
                    e = cudaStreamEndCapture(s, &graph);
                    if (ec != cudaSuccess) e = ec;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        }
        double ep_loss = 0.0;
        if (e == cudaSuccess) ep_loss = read_loss(s, ws, nblk, (long long)B * kMlpOut, &e);
        history.push_back(ep_loss);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(hyper);
    cudaFree(tstep);
    if (e == cudaSuccess) e = ws.check(s);
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
