// FP64 vector kernels of GMRES outside the device-resident Arnoldi step
// (krylov.cu): segmented dot products (one segment per problem), segmented
// scaling, linear combinations.  A basis of k vectors is stored with leading
// dimension ld.
#include <algorithm>

#include "common.h"

namespace sbie {

// out = a x + b y; y may alias out (axpy), so neither is __restrict__.
__global__ void lincomb_kernel(double a, const double* x, double b, const double* y, double* out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

static unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t blas_lincomb(sbie_ctx* c, double a, const double* x, double b, const double* y, double* out, long long n) {
    lincomb_kernel<<<grid_for(n), 256, 0, c->stream>>>(a, x, b, y, out, n); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t blas_axpy(sbie_ctx* c, double a, const double* x, double* y, long long n) {
    return blas_lincomb(c, a, x, 1.0, y, y, n);
}

// ---- segmented versions: the vector holds independent problems; segment p
// covers [seg[p], seg[p+1]) and node i / 3 belongs to problem node_prob[i / 3].

// partial[(j * P + p) * B + b] = sum over chunk b of segment p of V_j . w
__global__ void seg_dots_partial(const double* __restrict__ V, long long ld, const double* __restrict__ w,
                                 const long long* __restrict__ seg, int P, double* __restrict__ partial) {
    __shared__ double sh[32];
    const int B = gridDim.x, b = blockIdx.x, j = blockIdx.y, p = blockIdx.z;
    const long long s0 = seg[p], s1 = seg[p + 1];
    const double* v = V + (size_t)j * ld;
    double s = 0.0;
    for (long long i = s0 + (long long)b * blockDim.x + threadIdx.x; i < s1; i += (long long)B * blockDim.x)
        s = fma(v[i], w[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) partial[((size_t)j * P + p) * B + b] = s;
    }
}

__global__ void seg_dots_final(const double* __restrict__ partial, int B, int n, double* __restrict__ out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += partial[(size_t)q * B + b];
    out[q] = s;
}

// y[i] = scale[p(i)] * x[i]  (x may alias y)
__global__ void seg_scale_kernel(const double* x, const double* __restrict__ scale, const int* __restrict__ node_prob,
                                 double* y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = scale[node_prob[i / 3]] * x[i];
}

int seg_blocks(long long n3, int P) {
    long long per = (n3 + P - 1) / P;
    long long b = (per + 8191) / 8192;
    return (int)std::max<long long>(1, std::min<long long>(b, 128));
}

cudaError_t seg_dots(sbie_ctx* c, const double* V, int k, long long ld, const double* w, long long n3,
                     const long long* d_seg, int P, double* d_out) {
    const int B = seg_blocks(n3, P);
    if (!c->d_red || !d_out || (size_t)k * P * B > c->red_cap) return cudaErrorInvalidValue;
    dim3 grid(B, k, P);
    seg_dots_partial<<<grid, 256, 0, c->stream>>>(V, ld, w, d_seg, P, c->d_red); ++c->n_launch;
    const int n = k * P;
    seg_dots_final<<<(n + 255) / 256, 256, 0, c->stream>>>(c->d_red, B, n, d_out); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t seg_scale(sbie_ctx* c, const double* x, const double* d_scale, const int* d_node_prob, double* y,
                      long long n3) {
    seg_scale_kernel<<<grid_for(n3), 256, 0, c->stream>>>(x, d_scale, d_node_prob, y, n3); ++c->n_launch;
    return cudaGetLastError();
}

}  // namespace sbie
