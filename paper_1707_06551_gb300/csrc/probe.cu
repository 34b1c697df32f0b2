// FP32 throughput probe: the measured denominator of the far-field kernel's
// ALU roofline.  The paper has no counterpart; it measures the GPU.
//
// Every thread runs kChains independent packed FP32x2 fused multiply-add
// chains (FFMA2, two FMAs of one instruction: the instruction the far-field
// pair kernel is built on) for `iters` steps; the grid fills every SM with
// several resident CTAs.  FLOP = threads x iters x kChains x 4.  The chains'
// results are written so that the compiler keeps every operation.
#include "common.h"

namespace sbie {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma2_probe_kernel(int iters, float2 a, float2 b, float* out) {
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = make_float2(threadIdx.x * 1e-7f + c, c * 1e-3f);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = __ffma2_rn(acc[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c].x + acc[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace sbie

extern "C" sbie_status sphere_bie_fp32_peak_probe(double* tflops, double* ms) {
    using namespace sbie;
    if (!tflops) return SBIE_ERR_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("probe: ") + cudaGetErrorString(e));
        return SBIE_ERR_CUDA;
    }
    const int threads = 256, blocks = sms * 8, iters = 4096;
    float* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, sizeof(float) * threads * blocks);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    const float2 a = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch warms up
        cudaEventRecord(e0, s);
        ffma2_probe_kernel<<<blocks, threads, 0, s>>>(iters, a, b, out);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) best = std::min(best, t);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        set_last_error(std::string("probe: ") + cudaGetErrorString(e));
        return SBIE_ERR_CUDA;
    }
    const double flop = (double)threads * blocks * iters * 8.0 * kChains * 4.0;
    *tflops = flop / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return SBIE_OK;
}
