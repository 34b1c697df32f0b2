// Internal declarations of the pair network (mlp.cu) and the learned
// preconditioner (precond.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

namespace sbie {

constexpr int kPrecL = 4;                                  // low modes: VSH degree <= 4
constexpr int kLowModes = 3 * (kPrecL + 1) * (kPrecL + 1) - 2;  // 73 real coefficients per sphere
constexpr int kMlpIn = 5, kMlpHidden = 128, kMlpOut = kLowModes * kLowModes;

struct MlpLayout {
    int din[4], dout[4];
    long long w[4], b[4];  // offsets of the (din x dout) weights and (dout) biases
    long long total;
};
MlpLayout mlp_layout();

struct MlpTrainOpts {
    int epochs = 40;
    int batch = 256;
    double lr = 2e-3;
    unsigned long long seed = 7;
};

void mlp_init(unsigned long long seed, std::vector<float>& params);
cudaError_t mlp_train(const MlpTrainOpts& o, int n, const float* h_X, const float* h_T, float* h_params,
                      std::vector<double>& history);
cudaError_t mlp_gradients(const float* h_params, int n, const float* h_X, const float* h_T, float* h_grad,
                          double* loss);
cudaError_t mlp_to_bf16(cudaStream_t s, const float* w, __nv_bfloat16* wb);
cudaError_t mlp_forward_dev(cudaStream_t s, const float* w, const __nv_bfloat16* wb, int n, const float* X, float* Y);

// TF32 high part of x: round to nearest (ties away) at 10 explicit mantissa
// bits; x - tf32_hi(x) is exact in FP32.
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Epilogue of tc_gemm_tf32: C[n ldc + m] = sum_k A[m][k] B[n][k], then
// + bias[m] (kBias), tanh(. + bias[m]) (kBiasTanh) or x (1 - G[n ldg + m]^2)
// (kDTanh).
struct TcEpi {
    enum Mode { kNone = 0, kBias = 1, kBiasTanh = 2, kDTanh = 3 };
    float* C = nullptr;
    long long ldc = 0;
    const float* bias = nullptr;
    const float* G = nullptr;
    long long ldg = 0;
    int mode = kNone;
};
// 3xTF32 GEMM on the tensor cores (selfgemm.cu); a null Alo or Blo marks that
// operand exact in TF32 (not both); *err is set to 1 when one of its bounded
// waits runs out.  `work` (work_cap floats, or null) holds the partial sums of
// a split K.
cudaError_t tc_gemm_tf32(cudaStream_t s, int M, int N, int Kpad, const float* Ahi, const float* Alo,
                         const float* Bhi, const float* Blo, const TcEpi& ep, int* err, float* work = nullptr,
                         size_t work_cap = 0);

}  // namespace sbie
