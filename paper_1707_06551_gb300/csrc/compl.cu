// Rank-6-per-sphere terms and small per-sphere kernels:
//  - moments  M0_k = int psi, M1_k = int (y - c_k) x psi (node quadrature, Eq. 4.4);
//  - completion flow N (Eq. 5.19): Stokeslet (Eq. 2.19) of strength M0_k plus
//    rotlet M1_k x r / (8 pi |r|^3) at every centre, evaluated at every node;
//  - L_k of Eq. 5.8 on the own sphere and the nodal 1/2 I of Eqs. 5.8 / 5.19;
//  - rho of the mobility problem, the rigid projection of a surface velocity
//    and the resistance right-hand side;
//  - node geometry (Eq. 4.2) at create time.
#include "common.h"

namespace sbie {

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

// mode 0: moments of dens (weights from x64.w) -> mom[k][6]
// mode 1: rigid projection of dens -> vel[k], omega[k]
__global__ void sphere_reduce_kernel(const double* __restrict__ dens, const double* __restrict__ x64,
                                     const double* __restrict__ c, const double* __restrict__ a, int npn,
                                     int mode, double* __restrict__ o1, double* __restrict__ o2) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    double s[6] = {0, 0, 0, 0, 0, 0};
    const double cx = c[3 * k], cy = c[3 * k + 1], cz = c[3 * k + 2];
    for (int q = threadIdx.x; q < npn; q += blockDim.x) {
        long long i = (long long)k * npn + q;
        double w = x64[4 * i + 3];
        double dx = x64[4 * i] - cx, dy = x64[4 * i + 1] - cy, dz = x64[4 * i + 2] - cz;
        double fx = dens[3 * i] * w, fy = dens[3 * i + 1] * w, fz = dens[3 * i + 2] * w;
        s[0] += fx; s[1] += fy; s[2] += fz;
        s[3] += dy * fz - dz * fy;
        s[4] += dz * fx - dx * fz;
        s[5] += dx * fy - dy * fx;
    }
    double r[6];
    for (int d = 0; d < 6; ++d) r[d] = block_sum(s[d], sh);
    if (threadIdx.x == 0) {
        if (mode == 0) {
            for (int d = 0; d < 6; ++d) o1[6 * k + d] = r[d];
        } else {
            double ak = a[k];
            double f0 = 1.0 / (4.0 * kPi * ak * ak), f1 = 3.0 / (8.0 * kPi * ak * ak * ak * ak);
            for (int d = 0; d < 3; ++d) {
                o1[3 * k + d] = f0 * r[d];
                o2[3 * k + d] = f1 * r[3 + d];
            }
        }
    }
}

// 1 / sqrt(r2): IEEE in FP64; in FP32 the hardware reciprocal square root
// (a few ulp), the accuracy of the rest of the FP32 operator.
__device__ __forceinline__ double inv_sqrt(double r2) { return 1.0 / sqrt(r2); }
__device__ __forceinline__ float inv_sqrt(float r2) { return rsqrtf(r2); }

__device__ __forceinline__ void load12(const float* p, float (&v)[12]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float4 t = q[i];
        v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
}
__device__ __forceinline__ void load12(const double* p, double (&v)[12]) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double2 t = q[i];
        v[2 * i] = t.x; v[2 * i + 1] = t.y;
    }
}

// FP64: direct.  FP32: target and centre positions are split into float hi +
// lo parts so that x - c keeps relative FP32 accuracy (as in the far field).
template <typename T>
__global__ void completion_kernel(const double* __restrict__ x64, const double* __restrict__ c,
                                  const double* __restrict__ mom, const int* __restrict__ sph,
                                  const int* __restrict__ sph_prob, const int* __restrict__ prob_sph, long long N,
                                  double* __restrict__ out) {
    // out[i] += sum over spheres k of i's problem of
    //           G(x_i - c_k) M0_k + M1_k x (x_i - c_k) / (8 pi |x_i - c_k|^3)
    constexpr int TILE = 128;
    __shared__ __align__(16) T sd[TILE][12];  // centre hi (3), lo (3), force (3), torque (3)
    __shared__ int range[2];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < N;
    const long long ii = valid ? i : 0;
    const int pr = sph_prob[sph[ii]];
    const int k0 = prob_sph[pr], k1 = prob_sph[pr + 1];
    if (threadIdx.x == 0) {
        long long last = min(N - 1, (long long)blockIdx.x * blockDim.x + blockDim.x - 1);
        range[0] = k0;
        range[1] = prob_sph[sph_prob[sph[last]] + 1];
    }
    __syncthreads();
    const int kb = range[0], ke = range[1];
    const double X = x64[4 * ii], Y = x64[4 * ii + 1], Z = x64[4 * ii + 2];
    const T xh = (T)X, yh = (T)Y, zh = (T)Z;
    const T xl = (T)(X - (double)xh), yl = (T)(Y - (double)yh), zl = (T)(Z - (double)zh);
    T ux = 0, uy = 0, uz = 0;
    for (int b = kb; b < ke; b += TILE) {
        __syncthreads();
        for (int j = threadIdx.x; j < TILE; j += blockDim.x) {
            int k = b + j;
            for (int d = 0; d < 3; ++d) {
                double cd = (k < ke) ? c[3 * k + d] : 0.0;
                T h = (T)cd;
                sd[j][d] = h;
                sd[j][3 + d] = (T)(cd - (double)h);
            }
            for (int d = 0; d < 6; ++d) sd[j][6 + d] = (k < ke) ? (T)mom[6 * k + d] : (T)0;
        }
        __syncthreads();
        // this target's problem's spheres within the tile
        const int j0 = max(0, k0 - b), j1 = min(min(TILE, ke - b), k1 - b);
        for (int j = j0; j < j1; ++j) {
            T v[12];
            load12(sd[j], v);  // vector loads of the staged sphere (all threads read the same one)
            T dx = (xh - v[0]) + (xl - v[3]);
            T dy = (yh - v[1]) + (yl - v[4]);
            T dz = (zh - v[2]) + (zl - v[5]);
            T r2 = dx * dx + dy * dy + dz * dz;
            T ri = inv_sqrt(r2);
            T ri3 = ri * ri * ri;
            T fx = v[6], fy = v[7], fz = v[8];
            T tx = v[9], ty = v[10], tz = v[11];
            T rf = dx * fx + dy * fy + dz * fz;
            // Stokeslet f / r + r (r.f) / r^3 and rotlet (t x r) / r^3, common factor 1/(8 pi)
            ux += fx * ri + dx * rf * ri3 + (ty * dz - tz * dy) * ri3;
            uy += fy * ri + dy * rf * ri3 + (tz * dx - tx * dz) * ri3;
            uz += fz * ri + dz * rf * ri3 + (tx * dy - ty * dx) * ri3;
        }
    }
    if (valid) {
        const double f = 1.0 / (8.0 * kPi);
        out[3 * i] += f * (double)ux;
        out[3 * i + 1] += f * (double)uy;
        out[3 * i + 2] += f * (double)uz;
    }
}

// op 3 (mobility): out += 1/2 dens + M0_k + M1_k x (x - c_k) on own sphere
// op 4 (resistance): out += 1/2 dens
__global__ void finalize_kernel(int op, const double* __restrict__ dens, const double* __restrict__ x64,
                                const double* __restrict__ c, const double* __restrict__ mom, int npn,
                                long long N, double* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double o0 = 0.5 * dens[3 * i], o1 = 0.5 * dens[3 * i + 1], o2 = 0.5 * dens[3 * i + 2];
    if (op == (int)SBIE_OP_MOBILITY) {
        int k = (int)(i / npn);
        const double* M = mom + 6 * k;
        double dx = x64[4 * i] - c[3 * k], dy = x64[4 * i + 1] - c[3 * k + 1], dz = x64[4 * i + 2] - c[3 * k + 2];
        o0 += M[0] + (M[4] * dz - M[5] * dy);
        o1 += M[1] + (M[5] * dx - M[3] * dz);
        o2 += M[2] + (M[3] * dy - M[4] * dx);
    }
    out[3 * i] += o0;
    out[3 * i + 1] += o1;
    out[3 * i + 2] += o2;
}

__global__ void rho_kernel(const double* __restrict__ F, const double* __restrict__ T, const double* __restrict__ x64,
                           const double* __restrict__ c, const double* __restrict__ a, int npn, long long N,
                           double* __restrict__ rho) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = (int)(i / npn);
    double ak = a[k];
    double f0 = 1.0 / (4.0 * kPi * ak * ak), f1 = 3.0 / (8.0 * kPi * ak * ak * ak * ak);
    double dx = x64[4 * i] - c[3 * k], dy = x64[4 * i + 1] - c[3 * k + 1], dz = x64[4 * i + 2] - c[3 * k + 2];
    const double* t = T + 3 * k;
    rho[3 * i] = f0 * F[3 * k] + f1 * (t[1] * dz - t[2] * dy);
    rho[3 * i + 1] = f0 * F[3 * k + 1] + f1 * (t[2] * dx - t[0] * dz);
    rho[3 * i + 2] = f0 * F[3 * k + 2] + f1 * (t[0] * dy - t[1] * dx);
}

__global__ void rigid_split_kernel(const double* __restrict__ dens, const double* __restrict__ mom,
                                   const double* __restrict__ x64, const double* __restrict__ c,
                                   const double* __restrict__ a, int npn, long long N, double* __restrict__ q,
                                   double* __restrict__ r) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = (int)(i / npn);
    double ak = a[k];
    double f0 = 1.0 / (4.0 * kPi * ak * ak), f1 = 3.0 / (8.0 * kPi * ak * ak * ak * ak);
    double dx = x64[4 * i] - c[3 * k], dy = x64[4 * i + 1] - c[3 * k + 1], dz = x64[4 * i + 2] - c[3 * k + 2];
    const double* M = mom + 6 * k;  // int mu, int (y - c) x mu
    const double r0 = f0 * M[0] + f1 * (M[4] * dz - M[5] * dy);
    const double r1 = f0 * M[1] + f1 * (M[5] * dx - M[3] * dz);
    const double r2 = f0 * M[2] + f1 * (M[3] * dy - M[4] * dx);
    r[3 * i] = r0;
    r[3 * i + 1] = r1;
    r[3 * i + 2] = r2;
    q[3 * i] = dens[3 * i] - r0;
    q[3 * i + 1] = dens[3 * i + 1] - r1;
    q[3 * i + 2] = dens[3 * i + 2] - r2;
}

__global__ void res_rhs_kernel(const double* __restrict__ v, const double* __restrict__ w, double u0x, double u0y,
                               double u0z, double g00, double g01, double g02, double g10, double g11, double g12,
                               double g20, double g21, double g22, const double* __restrict__ x64,
                               const double* __restrict__ c, int npn, long long N, double* __restrict__ b) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = (int)(i / npn);
    double X = x64[4 * i], Y = x64[4 * i + 1], Z = x64[4 * i + 2];
    double dx = X - c[3 * k], dy = Y - c[3 * k + 1], dz = Z - c[3 * k + 2];
    const double* om = w + 3 * k;
    b[3 * i] = v[3 * k] + (om[1] * dz - om[2] * dy) - (u0x + g00 * X + g01 * Y + g02 * Z);
    b[3 * i + 1] = v[3 * k + 1] + (om[2] * dx - om[0] * dz) - (u0y + g10 * X + g11 * Y + g12 * Z);
    b[3 * i + 2] = v[3 * k + 2] + (om[0] * dy - om[1] * dx) - (u0z + g20 * X + g21 * Y + g22 * Z);
}

__global__ void geometry_kernel(const double* __restrict__ tab, TabLayout tl, const double* __restrict__ c,
                                const double* __restrict__ a, int n, double* __restrict__ x64,
                                float4* __restrict__ xhi, float4* __restrict__ xlo, float4* __restrict__ nrm,
                                double* __restrict__ nrm64, int* __restrict__ sph) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)n * tl.npn;
    if (i >= N) return;
    int k = (int)(i / tl.npn), q = (int)(i - (long long)k * tl.npn);
    int j = q / tl.nlon, l = q - j * tl.nlon;
    double ct = tab[tl.o_ct + j], st = tab[tl.o_st + j], cp = tab[tl.o_cph + l], sp = tab[tl.o_sph + l];
    double ex = st * cp, ey = st * sp, ez = ct;
    double ak = a[k];
    double X = c[3 * k] + ak * ex, Y = c[3 * k + 1] + ak * ey, Z = c[3 * k + 2] + ak * ez;
    double w = ak * ak * tab[tl.o_w + j];
    x64[4 * i] = X; x64[4 * i + 1] = Y; x64[4 * i + 2] = Z; x64[4 * i + 3] = w;
    float hx = (float)X, hy = (float)Y, hz = (float)Z;
    xhi[i] = make_float4(hx, hy, hz, (float)w);
    xlo[i] = make_float4((float)(X - (double)hx), (float)(Y - (double)hy), (float)(Z - (double)hz), 0.f);
    nrm[i] = make_float4((float)ex, (float)ey, (float)ez, 0.f);
    nrm64[4 * i] = ex; nrm64[4 * i + 1] = ey; nrm64[4 * i + 2] = ez; nrm64[4 * i + 3] = 0.0;
    sph[i] = k;
}

static unsigned nblk(long long n, int th) { return (unsigned)((n + th - 1) / th); }

cudaError_t launch_moments(sbie_ctx* c, const double* dens) {
    sphere_reduce_kernel<<<c->n, 256, 0, c->stream>>>(dens, c->d_x, c->d_c, c->d_a, c->npn, 0, c->d_mom, nullptr); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_completion(sbie_ctx* c, bool f32, double* out) {
    if (f32) {
        completion_kernel<float><<<nblk(c->N, 128), 128, 0, c->stream>>>(c->d_x, c->d_c, c->d_mom, c->d_sph,
                                                                          c->d_sph_prob, c->d_prob_sph, c->N, out);
    } else {
        completion_kernel<double><<<nblk(c->N, 128), 128, 0, c->stream>>>(c->d_x, c->d_c, c->d_mom, c->d_sph,
                                                                           c->d_sph_prob, c->d_prob_sph, c->N, out);
    }
    ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_finalize(sbie_ctx* c, int op, const double* dens, double* out) {
    finalize_kernel<<<nblk(c->N, 256), 256, 0, c->stream>>>(op, dens, c->d_x, c->d_c, c->d_mom, c->npn, c->N, out); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_rho(sbie_ctx* c, const double* F, const double* T, double* rho) {
    rho_kernel<<<nblk(c->N, 256), 256, 0, c->stream>>>(F, T, c->d_x, c->d_c, c->d_a, c->npn, c->N, rho); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_rigid_split(sbie_ctx* c, const double* dens, double* q, double* r) {
    rigid_split_kernel<<<nblk(c->N, 256), 256, 0, c->stream>>>(dens, c->d_mom, c->d_x, c->d_c, c->d_a, c->npn, c->N, q,
                                                               r); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_rigid_projection(sbie_ctx* c, const double* u, double* vel, double* omega) {
    sphere_reduce_kernel<<<c->n, 256, 0, c->stream>>>(u, c->d_x, c->d_c, c->d_a, c->npn, 1, vel, omega); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_resistance_rhs(sbie_ctx* c, const double* vel, const double* omega, const double* u0,
                                  const double* G, double* b) {
    double z[3] = {0, 0, 0}, g0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double* U = u0 ? u0 : z;
    const double* g = G ? G : g0;
    res_rhs_kernel<<<nblk(c->N, 256), 256, 0, c->stream>>>(vel, omega, U[0], U[1], U[2], g[0], g[1], g[2], g[3], g[4],
                                                           g[5], g[6], g[7], g[8], c->d_x, c->d_c, c->npn, c->N, b); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_geometry(sbie_ctx* c) {
    geometry_kernel<<<nblk(c->N, 256), 256, 0, c->stream>>>(c->d_tab, c->tl, c->d_c, c->d_a, c->n, c->d_x, c->d_xhi,
                                                            c->d_xlo, c->d_nrm, c->d_nrm64, c->d_sph); ++c->n_launch;
    return cudaGetLastError();
}

}  // namespace sbie
