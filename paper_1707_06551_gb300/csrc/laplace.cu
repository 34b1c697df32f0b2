// Laplace layer potentials on N spheres (Sec. 2.2, Eq. 2.18; Sec. 3.1, Eqs.
// 3.3-3.5 and Theorem 1; the flux of Sec. 3.3, Eqs. 3.13-3.16) for the
// magnetostatic problem of the multiphysics case study (Problem 3, Eqs.
// 5.9-5.13).  Scalar densities live in component 0 of the context's [N][3]
// vectors (stride 3), so the GMRES machinery serves them unchanged.
//
//   S^L[q](x) = sum_y q w / (4 pi |x - y|),   D^L[m](x) = sum_y m w n(y).(x - y) / (4 pi |x - y|^3),
//   K^L[q](x) = n(x) . grad S^L[q](x),        grad S^L[q](x) = -sum_y q w (x - y) / (4 pi |x - y|^3).
//
// Self term (one CTA per sphere, FP64): DFT in phi, Gauss-Legendre contraction
// to the scalar coefficients c_nm, the Theorem 1 signature -- S^L a/(2n+1); D^L
// and K^L the principal value -1/(2(2n+1)) (K+ = D-, K- = D+) -- and synthesis;
// for the exterior gradient of S^L the synthesis is the V-mode field
// sum c_nm V_n^m / (2n+1) (Eq. 3.3 differentiated, scale free).
// Far field: the smooth quadrature of Eq. 4.4 over every node of every sphere
// that is neither the target sphere nor a close partner (FP64, one thread per
// target node, sources staged through shared memory; excluded sources are moved
// far away with zero weight, as in the Stokes kernels).
// Close pairs: the exterior expansions of Eqs. 3.3-3.4 evaluated by the solid
// harmonic kernels of near.cu (launch_near_laplace).
#include "common.h"

namespace sbie {

namespace {

struct LapSelfArgs {
    int p, nlat, nlon, npn;
    TabLayout tl;
    const double* tab;
    const double* q;   // component 0 of [N][3]
    double* out;       // scalar modes: component 0 of [N][3]; gradient: [N][3]
    const double* radius;
    double* coef;      // [n][P1 (n)][P1 (m)][2] or nullptr
    int mode;          // kLap*
    int accumulate;
};

__global__ void laplace_self_kernel(LapSelfArgs A) {
    const int s = blockIdx.x;
    const int p = A.p, P1 = p + 1, nlat = A.nlat, nlon = A.nlon, npn = A.npn;
    const TabLayout& tl = A.tl;
    const double* __restrict__ tab = A.tab;
    const double* ct = tab + tl.o_ct;
    const double* st = tab + tl.o_st;
    const double* wq = tab + tl.o_w;
    const double* cph = tab + tl.o_cph;
    const double* sph = tab + tl.o_sph;
    const double* cmk = tab + tl.o_cmk;
    const double* smk = tab + tl.o_smk;
    const double* Pt = tab + tl.o_P;
    const double* dPt = tab + tl.o_dP;
    const double* mSt = tab + tl.o_mS;
    const bool grad = A.mode == kLapGrad;
    const int nc = grad ? 3 : 1;

    extern __shared__ double sm[];
    double* f = sm;                        // [3][npn]
    double* Fh = f + 3 * npn;              // [3][nlat][P1][2]
    double* cf = Fh + 3 * nlat * P1 * 2;   // [P1 (n)][P1 (m)][2]
    const int tid = threadIdx.x, bd = blockDim.x;
    const size_t base = (size_t)s * npn;

    for (int q = tid; q < npn; q += bd) f[q] = A.q[(base + q) * 3];
    __syncthreads();
    // DFT in phi: Fh[j][m] = sum_k f e^{-i m phi_k}
    for (int q = tid; q < nlat * P1; q += bd) {
        const int j = q / P1, m = q - j * P1;
        const double* row = f + j * nlon;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < nlon; ++k) {
            re = fma(row[k], cmk[m * nlon + k], re);
            im = fma(-row[k], smk[m * nlon + k], im);
        }
        Fh[2 * q] = re;
        Fh[2 * q + 1] = im;
    }
    __syncthreads();
    // Legendre contraction, coefficients, signature
    const double a = A.radius[s];
    for (int q = tid; q < P1 * P1; q += bd) {
        const int n = q / P1, m = q - n * P1;
        double cr = 0.0, ci = 0.0;
        if (m <= n) {
            for (int j = 0; j < nlat; ++j) {
                const double w = wq[j] * Pt[(m * P1 + n) * nlat + j];
                cr = fma(w, Fh[2 * (j * P1 + m)], cr);
                ci = fma(w, Fh[2 * (j * P1 + m) + 1], ci);
            }
            if (m == 0) ci = 0.0;
        }
        if (A.coef) {
            double* cg = A.coef + (size_t)s * P1 * P1 * 2;
            cg[2 * q] = cr;
            cg[2 * q + 1] = ci;
        }
        const double t = 1.0 / (2.0 * n + 1.0);
        const double sig = A.mode == kLapSL ? a * t : (grad ? t : -0.5 * t);
        cf[2 * q] = sig * cr;
        cf[2 * q + 1] = sig * ci;
    }
    __syncthreads();
    // inverse Legendre: scalar A(j, m) = sum_n b P; gradient (r, theta, phi)
    // components sum_n b (-(n+1) P, dP, i mS)
    for (int q = tid; q < nc * nlat * P1; q += bd) {
        const int c = q / (nlat * P1), rem = q - c * nlat * P1, j = rem / P1, m = rem - j * P1;
        double ar = 0.0, ai = 0.0;
        for (int n = m; n <= p; ++n) {
            const int o = (m * P1 + n) * nlat + j;
            const double br = cf[2 * (n * P1 + m)], bi = cf[2 * (n * P1 + m) + 1];
            if (c == 0) {
                const double P = grad ? -(n + 1.0) * Pt[o] : Pt[o];
                ar = fma(br, P, ar);
                ai = fma(bi, P, ai);
            } else if (c == 1) {
                ar = fma(br, dPt[o], ar);
                ai = fma(bi, dPt[o], ai);
            } else {  // i b mS
                ar = fma(-bi, mSt[o], ar);
                ai = fma(br, mSt[o], ai);
            }
        }
        Fh[2 * q] = ar;
        Fh[2 * q + 1] = ai;
    }
    __syncthreads();
    // inverse DFT
    for (int q = tid; q < nc * npn; q += bd) {
        const int c = q / npn, r = q - c * npn, j = r / nlon, k = r - j * nlon;
        const double* av = Fh + 2 * ((c * nlat + j) * P1);
        double v = 0.0;
        for (int m = 1; m <= p; ++m) {
            v = fma(av[2 * m], cmk[m * nlon + k], v);
            v = fma(-av[2 * m + 1], smk[m * nlon + k], v);
        }
        f[q] = av[0] + 2.0 * v;
    }
    __syncthreads();
    for (int q = tid; q < npn; q += bd) {
        double* o = A.out + (base + q) * 3;
        if (!grad) {
            o[0] = A.accumulate ? o[0] + f[q] : f[q];
            continue;
        }
        const int j = q / nlon, k = q - j * nlon;
        const double c = ct[j], sn = st[j], cp = cph[k], sp = sph[k];
        const double fr = f[q], ft = f[npn + q], fp = f[2 * npn + q];
        const double gx = fr * sn * cp + ft * c * cp - fp * sp;
        const double gy = fr * sn * sp + ft * c * sp + fp * cp;
        const double gz = fr * c - ft * sn;
        if (A.accumulate) {
            o[0] += gx; o[1] += gy; o[2] += gz;
        } else {
            o[0] = gx; o[1] = gy; o[2] = gz;
        }
    }
}

constexpr int kLapTile = 256;

// One thread per target node, CTA = (target sphere, chunk of its nodes).
__global__ void __launch_bounds__(256) laplace_far_kernel(int npn, int chunks, int mode, const double* __restrict__ q,
                                                         const double* __restrict__ x64,
                                                         const double* __restrict__ nrm64,
                                                         const int* __restrict__ sph,
                                                         const int* __restrict__ near_ptr,
                                                         const int* __restrict__ near_idx,
                                                         const int* __restrict__ sph_prob,
                                                         const int* __restrict__ prob_sph, int n, double* out) {
    const int sphere = blockIdx.x / chunks, chunk = blockIdx.x - sphere * chunks;
    extern __shared__ double4 lsm[];
    double4* sp = lsm;                // position, weight x density
    double4* sn = lsm + kLapTile;     // source normal
    unsigned* flags = reinterpret_cast<unsigned*>(lsm + 2 * kLapTile);
    const int words = (n + 31) / 32;
    for (int w = threadIdx.x; w < words; w += blockDim.x) flags[w] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicOr(&flags[sphere >> 5], 1u << (sphere & 31));
        for (int e = near_ptr[sphere]; e < near_ptr[sphere + 1]; ++e) {
            const int k = near_idx[e];
            atomicOr(&flags[k >> 5], 1u << (k & 31));
        }
    }
    const int tq = chunk * blockDim.x + threadIdx.x;
    const bool valid = tq < npn;
    const long long node = (long long)sphere * npn + (valid ? tq : npn - 1);
    const double tx = x64[4 * node], ty = x64[4 * node + 1], tz = x64[4 * node + 2];
    const double nx = nrm64[4 * node], ny = nrm64[4 * node + 1], nz = nrm64[4 * node + 2];
    const int pr = sph_prob[sphere];
    const long long b0 = (long long)prob_sph[pr] * npn, b1 = (long long)prob_sph[pr + 1] * npn;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const double far_off = 1.0e6;
    for (long long base = b0; base < b1; base += kLapTile) {
        __syncthreads();
        for (int j = threadIdx.x; j < kLapTile; j += blockDim.x) {
            const long long s = base + j;
            double4 P = make_double4(tx + far_off, ty + far_off, tz + far_off, 0.0);
            double4 Nn = make_double4(0.0, 0.0, 0.0, 0.0);
            if (s < b1) {
                const int k = sph[s];
                if (!((flags[k >> 5] >> (k & 31)) & 1u)) {
                    P = make_double4(x64[4 * s], x64[4 * s + 1], x64[4 * s + 2], x64[4 * s + 3] * q[3 * s]);
                    if (mode == kLapDL) Nn = make_double4(nrm64[4 * s], nrm64[4 * s + 1], nrm64[4 * s + 2], 0.0);
                }
            }
            sp[j] = P;
            sn[j] = Nn;
        }
        __syncthreads();
        for (int j = 0; j < kLapTile; ++j) {
            const double4 P = sp[j];
            const double dx = tx - P.x, dy = ty - P.y, dz = tz - P.z;
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double ri = rsqrt(r2);
            if (mode == kLapSL) {
                a0 = fma(P.w, ri, a0);
            } else {
                const double w3 = P.w * ri * ri * ri;
                if (mode == kLapDL) {
                    const double4 Nn = sn[j];
                    a0 = fma(w3, fma(dz, Nn.z, fma(dy, Nn.y, dx * Nn.x)), a0);
                } else if (mode == kLapKL) {
                    a0 = fma(-w3, fma(dz, nz, fma(dy, ny, dx * nx)), a0);
                } else {
                    a0 = fma(-w3, dx, a0);
                    a1 = fma(-w3, dy, a1);
                    a2 = fma(-w3, dz, a2);
                }
            }
        }
    }
    if (!valid) return;
    const double s4 = 1.0 / (4.0 * kPi);
    double* o = out + node * 3;
    o[0] += s4 * a0;
    if (mode == kLapGrad) {
        o[1] += s4 * a1;
        o[2] += s4 * a2;
    }
}

__global__ void magnetic_finalize_kernel(long long N, double eta, const double* __restrict__ in,
                                         double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[3 * i] = 0.5 * in[3 * i] + eta * out[3 * i];
    out[3 * i + 1] = 0.5 * in[3 * i + 1];
    out[3 * i + 2] = 0.5 * in[3 * i + 2];
}

// b = (eta H0 . n, 0, 0) at every node
__global__ void magnetic_rhs_kernel(long long N, double eta, double hx, double hy, double hz,
                                    const double* __restrict__ nrm64, double* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    b[3 * i] = eta * (hx * nrm64[4 * i] + hy * nrm64[4 * i + 1] + hz * nrm64[4 * i + 2]);
    b[3 * i + 1] = 0.0;
    b[3 * i + 2] = 0.0;
}

// Maxwell traction (H.n) H - |H|^2 n / 2 with H = H0 - grad S^L[q] (in place)
__global__ void maxwell_traction_kernel(long long N, double hx, double hy, double hz,
                                        const double* __restrict__ nrm64, double* __restrict__ g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double H0 = hx - g[3 * i], H1 = hy - g[3 * i + 1], H2 = hz - g[3 * i + 2];
    const double n0 = nrm64[4 * i], n1 = nrm64[4 * i + 1], n2 = nrm64[4 * i + 2];
    const double hn = H0 * n0 + H1 * n1 + H2 * n2, hh = 0.5 * (H0 * H0 + H1 * H1 + H2 * H2);
    g[3 * i] = hn * H0 - hh * n0;
    g[3 * i + 1] = hn * H1 - hh * n1;
    g[3 * i + 2] = hn * H2 - hh * n2;
}

unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t laplace_apply(sbie_ctx* c, int mode, const double* q, double* out) {
    // self term writes `out` (component 0, or all three for the gradient)
    {
        StageScope st(c, ST_SELF);
        LapSelfArgs A;
        A.p = c->p; A.nlat = c->nlat; A.nlon = c->nlon; A.npn = c->npn;
        A.tl = c->tl; A.tab = c->d_tab; A.q = q; A.out = out; A.radius = c->d_a;
        A.coef = c->n_near > 0 ? c->d_lcoef : nullptr;
        A.mode = mode; A.accumulate = 0;
        const int P1 = c->p + 1;
        const size_t sm = sizeof(double) * (size_t)(3 * c->npn + 3 * c->nlat * P1 * 2 + P1 * P1 * 2);
        if (sm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(laplace_self_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 200 * 1024);
            if (e != cudaSuccess) return e;
        }
        laplace_self_kernel<<<c->n, 256, sm, c->stream>>>(A); ++c->n_launch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (c->far_pair_count > 0) {
        StageScope st(c, ST_FAR);
        const int th = (int)std::min<long long>(256, ((c->npn + 31) / 32) * 32);
        const int chunks = (c->npn + th - 1) / th;
        const size_t sm = 2 * kLapTile * sizeof(double4) + ((c->n + 31) / 32) * sizeof(unsigned);
        if (sm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(laplace_far_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
            if (e != cudaSuccess) return e;
        }
        laplace_far_kernel<<<c->n * chunks, th, sm, c->stream>>>(c->npn, chunks, mode, q, c->d_x, c->d_nrm64,
                                                                  c->d_sph, c->d_near_ptr, c->d_near_idx,
                                                                  c->d_sph_prob, c->d_prob_sph, c->n, out);
        ++c->n_launch;
        if (c->prof.on) c->prof.pairs_f64 += c->far_pair_count;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (c->n_near > 0) {
        StageScope st(c, ST_NEAR);
        return launch_near_laplace(c, mode, out);
    }
    return cudaSuccess;
}

cudaError_t launch_magnetic_finalize(sbie_ctx* c, double eta, const double* in, double* out) {
    magnetic_finalize_kernel<<<nblocks(c->N, 256), 256, 0, c->stream>>>(c->N, eta, in, out); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_magnetic_rhs(sbie_ctx* c, double eta, const double* H0, double* b) {
    magnetic_rhs_kernel<<<nblocks(c->N, 256), 256, 0, c->stream>>>(c->N, eta, H0[0], H0[1], H0[2], c->d_nrm64, b);
    ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_maxwell_traction(sbie_ctx* c, const double* H0, double* g) {
    maxwell_traction_kernel<<<nblocks(c->N, 256), 256, 0, c->stream>>>(c->N, H0[0], H0[1], H0[2], c->d_nrm64, g);
    ++c->n_launch;
    return cudaGetLastError();
}

}  // namespace sbie
