// Device-resident GMRES restart cycle.  The Arnoldi step (classical
// Gram-Schmidt applied twice), the Givens update of the Hessenberg least-
// squares problem and the per-problem convergence test all run on the GPU,
// with the Krylov index k held in device memory.  One iteration is captured
// once as the body of a CUDA graph WHILE node; the advance kernel sets the
// node's condition, so a whole cycle is one graph launch with no host round
// trip per iteration.  Without a graph (profiling, or use_graphs = 0) the
// host enqueues the same kernels one iteration at a time and reads the
// continue flag after each, so both drivers compute the same iterates.
#include <cmath>

#include "common.h"

namespace sbie {

namespace {

// st[0] = k, st[1] = iteration limit of the cycle, st[2] = continue, st[3] = non-finite flag,
// st[4] = some problem still iterating

__global__ void cycle_init_kernel(ArnoldiDev A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        A.st[0] = 0;
        A.st[1] = (int)A.pack[4 * A.P];
        A.st[2] = 1;
        A.st[3] = 0;
        A.st[4] = 1;
    }
    if (p >= A.P) return;
    const double nb = A.pack[p], tol = A.pack[A.P + p], beta = A.pack[2 * A.P + p];
    const bool act = A.pack[3 * A.P + p] != 0.0;
    A.nb[p] = nb;
    A.tol[p] = tol;
    A.live[p] = act ? 1 : 0;
    A.kd[p] = 0;
    double* g = A.g + (size_t)p * (A.m + 1);
    for (int j = 0; j <= A.m; ++j) g[j] = 0.0;
    g[0] = act ? beta : 0.0;
}

// dst = V_k
__global__ void copy_k_kernel(const double* __restrict__ V, long long ld, const int* __restrict__ st,
                              double* __restrict__ dst, long long n) {
    const double* v = V + (size_t)st[0] * ld;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = v[i];
}

// partial[(j P + p) B + b] = chunk b of segment p of V_j . w, for j <= k
__global__ void dots_dk_partial(const double* __restrict__ V, long long ld, const double* __restrict__ w,
                                const long long* __restrict__ seg, int P, const int* __restrict__ st,
                                double* __restrict__ partial) {
    const int B = gridDim.x, b = blockIdx.x, j = blockIdx.y, p = blockIdx.z;
    if (j > st[0]) return;
    __shared__ double sh[32];
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

// h[j P + p] = sum of the partials for j <= k; zero for problems that stopped
__global__ void dots_dk_final(const double* __restrict__ partial, int B, int P, const int* __restrict__ st,
                              const int* __restrict__ live, double* __restrict__ h) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (st[0] + 1) * P) return;
    const int p = q % P;
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += partial[(size_t)q * B + b];
    h[q] = live[p] ? s : 0.0;
}

// w[i] += sign sum_{j < count} h[j P + p(i)] V_j[i], count = k + incl
__global__ void gemv_dk_kernel(const double* __restrict__ V, long long ld, const double* __restrict__ h, int P,
                               double sign, const int* __restrict__ node_prob, const int* __restrict__ st, int incl,
                               double* __restrict__ w, long long n) {
    const int count = st[0] + incl;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int p = node_prob[i / 3];
        double s = 0.0;
        for (int j = 0; j < count; ++j) s = fma(h[(size_t)j * P + p], V[(size_t)j * ld + i], s);
        w[i] = fma(sign, s, w[i]);
    }
}

// Column k of each live problem's Hessenberg matrix: sum of the two Gram-
// Schmidt passes, previous rotations applied, new rotation from ||w||; the
// residual estimate |g_{k+1}| decides whether the problem stops.
__global__ void arnoldi_update_kernel(ArnoldiDev A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    const int k = A.st[0], m = A.m, P = A.P;
    if (!A.live[p]) {
        A.scale[p] = 0.0;
        return;
    }
    const double hk1 = sqrt(fmax(0.0, A.nrm[p]));
    if (!isfinite(hk1)) {
        atomicExch(A.st + 3, 1);
        A.live[p] = 0;
        A.scale[p] = 0.0;
        return;
    }
    A.scale[p] = hk1 > 0.0 ? 1.0 / hk1 : 0.0;
    double* H = A.H + (size_t)p * (m + 1) * m;
    double* cs = A.cs + (size_t)p * m;
    double* sn = A.sn + (size_t)p * m;
    double* g = A.g + (size_t)p * (m + 1);
    for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = A.h1[(size_t)j * P + p] + A.h2[(size_t)j * P + p];
    for (int j = 0; j < k; ++j) {
        const double a0 = H[(size_t)j * m + k], a1 = H[(size_t)(j + 1) * m + k];
        H[(size_t)j * m + k] = cs[j] * a0 + sn[j] * a1;
        H[(size_t)(j + 1) * m + k] = -sn[j] * a0 + cs[j] * a1;
    }
    const double hk = H[(size_t)k * m + k];
    const double den = hypot(hk, hk1);
    cs[k] = den > 0.0 ? hk / den : 1.0;
    sn[k] = den > 0.0 ? hk1 / den : 0.0;
    H[(size_t)k * m + k] = den;
    g[k + 1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    A.kd[p] = k + 1;
    if (fabs(g[k + 1]) / A.nb[p] <= A.tol[p] || hk1 == 0.0) A.live[p] = 0;
}

// k <- k + 1; the loop continues while a problem is live, the cycle has room
// and nothing non-finite was met.
__global__ void arnoldi_advance_kernel(ArnoldiDev A, cudaGraphConditionalHandle cond, int has_cond) {
    int any = 0;
    for (int p = threadIdx.x; p < A.P; p += blockDim.x) any |= A.live[p];
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        const int k1 = A.st[0] + 1;
        A.st[0] = k1;
        const int cont = (any && k1 < A.st[1] && A.st[3] == 0) ? 1 : 0;
        A.st[2] = cont;
        A.st[4] = any;
        if (has_cond) cudaGraphSetConditional(cond, cont);
    }
}

// V_k = scale[p] w (k already advanced)
__global__ void scale_to_k_kernel(const double* __restrict__ w, const double* __restrict__ scale,
                                  const int* __restrict__ node_prob, const int* __restrict__ st, double* __restrict__ V,
                                  long long ld, long long n) {
    double* v = V + (size_t)st[0] * ld;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = scale[node_prob[i / 3]] * w[i];
}

// y = H^{-1} g over the kd[p] leading columns (upper triangular), y[j P + p]
__global__ void lsq_kernel(ArnoldiDev A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    const int m = A.m, P = A.P, kk = A.kd[p];
    const double* H = A.H + (size_t)p * (m + 1) * m;
    const double* g = A.g + (size_t)p * (m + 1);
    for (int j = kk; j < m; ++j) A.y[(size_t)j * P + p] = 0.0;
    for (int i = kk - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < kk; ++j) s -= H[(size_t)i * m + j] * A.y[(size_t)j * P + p];
        A.y[(size_t)i * P + p] = s / H[(size_t)i * m + i];
    }
}

unsigned grid_n(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t arnoldi_cycle_init(sbie_ctx* c, const ArnoldiDev& A) {
    cycle_init_kernel<<<(A.P + 127) / 128, 128, 0, c->stream>>>(A); ++c->n_launch;
    return cudaGetLastError();
}

// One Arnoldi iteration on the device (the body of the captured loop).
// Apply is enqueued by the caller between copy_k and the Gram-Schmidt passes.
cudaError_t arnoldi_copy_k(sbie_ctx* c, const ArnoldiDev& A, const double* V, long long n3, double* dst) {
    copy_k_kernel<<<grid_n(n3), 256, 0, c->stream>>>(V, n3, A.st, dst, n3); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t arnoldi_orthogonalise(sbie_ctx* c, const ArnoldiDev& A, double* V, long long n3, const long long* d_seg,
                                  const int* d_node_prob) {
    const int B = seg_blocks(n3, A.P);
    if (!c->d_red || (size_t)(A.m + 1) * A.P * B > c->red_cap) return cudaErrorInvalidValue;
    for (int pass = 0; pass < 2; ++pass) {
        double* h = pass == 0 ? A.h1 : A.h2;
        dim3 grid(B, A.m, A.P);  // rows j <= k < m are live
        dots_dk_partial<<<grid, 256, 0, c->stream>>>(V, n3, A.w, d_seg, A.P, A.st, c->d_red); ++c->n_launch;
        dots_dk_final<<<(A.m * A.P + 255) / 256, 256, 0, c->stream>>>(c->d_red, B, A.P, A.st, A.live, h);
        ++c->n_launch;
        gemv_dk_kernel<<<grid_n(n3), 256, 0, c->stream>>>(V, n3, h, A.P, -1.0, d_node_prob, A.st, 1, A.w, n3);
        ++c->n_launch;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return seg_dots(c, A.w, 1, n3, A.w, n3, d_seg, A.P, A.nrm);
}

cudaError_t arnoldi_step_end(sbie_ctx* c, const ArnoldiDev& A, double* V, long long n3, const int* d_node_prob,
                             cudaGraphConditionalHandle cond, bool has_cond) {
    arnoldi_update_kernel<<<(A.P + 127) / 128, 128, 0, c->stream>>>(A); ++c->n_launch;
    arnoldi_advance_kernel<<<1, 256, 0, c->stream>>>(A, cond, has_cond ? 1 : 0); ++c->n_launch;
    scale_to_k_kernel<<<grid_n(n3), 256, 0, c->stream>>>(A.w, A.scale, d_node_prob, A.st, V, n3, n3); ++c->n_launch;
    return cudaGetLastError();
}

// After the cycle: y from the triangular systems, then out += sign V y over
// the k executed columns.
cudaError_t arnoldi_finish(sbie_ctx* c, const ArnoldiDev& A, const double* V, long long n3, const int* d_node_prob,
                           double* out) {
    lsq_kernel<<<(A.P + 127) / 128, 128, 0, c->stream>>>(A); ++c->n_launch;
    gemv_dk_kernel<<<grid_n(n3), 256, 0, c->stream>>>(V, n3, A.y, A.P, 1.0, d_node_prob, A.st, 0, out, n3);
    ++c->n_launch;
    return cudaGetLastError();
}

}  // namespace sbie
