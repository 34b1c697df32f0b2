// Close pairs (Sec. 4.1, "Singular and near-singular integrands"): the
// contribution of a close source sphere k to the nodes of target sphere i is
// the exterior expansion of k's density evaluated at those nodes -- S by
// Eqs. 3.6-3.8 (times the source radius), D by Eqs. 3.9-3.11 and the traction
// K of Eq. 3.18 with the single-layer pressure of Sec. 3.2.
//
// GPU formulation.  With I_nm = r^{-n-1} Y_n^m (an irregular solid harmonic),
//   V r^{-n-2} = grad I,   V r^{-n} = r^2 grad I,
//   W r^{-n}   = r^2 grad I + (2n+1) x I,   X r^{-n-1} = x cross grad I,
// so an exterior branch of Eqs. 3.6-3.11 is
//   u = grad Pa + r^2 grad Pb + x Pc + x cross grad Pd
// with harmonic Pa..Pd whose coefficients are the signature-weighted VSH
// coefficients; the S pressure of Sec. 3.2 is Pe = sum n phi^W I.  In the basis
// J_nm = P_n^m(cos th) e^{i m ph} / r^{n+1} the Cartesian derivatives are index
// shifts:  d_z J_nm = -(n-m+1) J_{n+1,m},  (d_x + i d_y) J_nm = -J_{n+1,m+1},
// (d_x - i d_y) J_nm = (n-m+1)(n-m+2) J_{n+1,m-1} (m >= 1).  near_prep turns a
// source sphere's coefficients into "channels" (the real coefficient vectors
// of grad Pa, ..., hess Pd, Pe); near_eval evaluates the J_nm at each target
// by their Cartesian recurrence (no angles, so no polar singularity) and
// contracts them with the channels.  The traction follows from the channels:
//   t = 2 Ha n + 2 (x.n) gb + 2 (gb.n) x + 2 r^2 Hb n + 2 Pc n + (gc.n) x
//       + (x.n) gc + x cross (Hd n) + Hd (n cross x) - Pe n.
#include "common.h"

namespace sbie {

struct NearArgs {
    int n, p, npn, L, nch, chunks, threads;
    const double* __restrict__ coef;   // [n][3][p+1][p+1][2]
    const float* __restrict__ coeff;   // the same in FP32 (near_prep reads it when coef is null)
    const double* __restrict__ radius;
    const double* __restrict__ c;
    const double* __restrict__ x64;    // [N][4]
    const double* __restrict__ nrm64;  // [N][4]
    const int* __restrict__ near_ptr;
    const int* __restrict__ near_idx;
    double* __restrict__ chan;         // [n][K][nch]
    float* __restrict__ chanf;         // [n][K][nchf]
    int nchf;
    int sel;                           // Laplace: 0 S^L value, 1 D^L value, 2 flux of S^L (KIND 3)
    double* __restrict__ out;          // [N][3]
};

// sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!)
__device__ __forceinline__ double ynorm(int n, int m) {
    double r = (2.0 * n + 1.0) / (4.0 * kPi);
    for (int k = n - m + 1; k <= n + m; ++k) r /= (double)k;
    return sqrt(r);
}

// Derivative of a real harmonic expansion (layout sh_index(L, .)) along axis
// d (0 = x, 1 = y, 2 = z), evaluated as a gather for output entry (n, m, part).
__device__ __forceinline__ double deriv_gather(const double* a, int L, int d, int n, int m, int part) {
    if (n == 0) return 0.0;
    const int n0 = n - 1;
    double v = 0.0;
    if (d == 2) {
        if (m <= n0) v = -(double)(n - m) * a[sh_index(L, n0, m, part)];
        return v;
    }
    // kappa(n0, m+1) = (n0 - m)(n0 - m + 1)
    const bool up = (m + 1 <= n0);
    const double kap = up ? (double)(n0 - m) * (double)(n0 - m + 1) : 0.0;
    if (d == 0) {
        if (part == 0) {
            if (m == 1) v -= a[sh_index(L, n0, 0, 0)];
            else if (m >= 2) v -= 0.5 * a[sh_index(L, n0, m - 1, 0)];
            if (up) v += 0.5 * kap * a[sh_index(L, n0, m + 1, 0)];
        } else {
            if (m >= 2) v -= 0.5 * a[sh_index(L, n0, m - 1, 1)];
            if (up) v += 0.5 * kap * a[sh_index(L, n0, m + 1, 1)];
        }
    } else {
        if (part == 0) {
            if (m >= 2) v += 0.5 * a[sh_index(L, n0, m - 1, 1)];
            if (up) v += 0.5 * kap * a[sh_index(L, n0, m + 1, 1)];
        } else {
            if (m == 1) v -= a[sh_index(L, n0, 0, 0)];
            else if (m >= 2) v -= 0.5 * a[sh_index(L, n0, m - 1, 0)];
            if (up) v -= 0.5 * kap * a[sh_index(L, n0, m + 1, 0)];
        }
    }
    return v;
}

// Apply derivative d to K-vector `src` -> `dst` (all entries), cooperative over the CTA.
__device__ void deriv_all(const double* src, double* dst, int L, int d) {
    for (int q = threadIdx.x; q < sh_count(L); q += blockDim.x) {
        // decode q -> (n, m, part)
        int m = 0, rem = q;
        if (rem <= L) {
            dst[q] = deriv_gather(src, L, d, rem, 0, 0);
            continue;
        }
        rem -= (L + 1);
        m = 1;
        while (rem >= 2 * (L + 1 - m)) {
            rem -= 2 * (L + 1 - m);
            ++m;
        }
        int n = m + rem / 2, part = rem & 1;
        dst[q] = deriv_gather(src, L, d, n, m, part);
    }
}

// Laplace close pairs (Eqs. 3.3-3.4): from the scalar coefficients c_nm of a
// source sphere ([P1 (n)][P1 (m)][2]), the channels
// [Phi_S, grad Phi_S (3), Phi_D] with Phi_S = sum c I_nm / (2n+1) and
// Phi_D = sum n c I_nm / (2n+1), I_nm = r^{-n-1} Y_n^m.
__global__ void near_prep_laplace_kernel(NearArgs A) {
    const int s = blockIdx.x;
    if (A.near_ptr[s + 1] == A.near_ptr[s]) return;
    const int p = A.p, P1 = p + 1, L = A.L, K = sh_count(L), nch = A.nch;
    extern __shared__ double sm[];
    double* phs = sm;         // [K]
    double* phd = sm + K;     // [K]
    double* grad = sm + 2 * K;  // [3][K]
    const double* cf = A.coef + (size_t)s * P1 * P1 * 2;
    for (int q = threadIdx.x; q < 2 * K; q += blockDim.x) sm[q] = 0.0;
    __syncthreads();
    for (int q = threadIdx.x; q < P1 * P1; q += blockDim.x) {
        const int n = q / P1, m = q - n * P1;
        if (m > n) continue;
        const double t = 1.0 / (2.0 * n + 1.0);
        const double cr = cf[2 * q], ci = cf[2 * q + 1];
        const double e = (m == 0 ? 1.0 : 2.0) * ynorm(n, m);
        const int ire = sh_index(L, n, m, 0);
        phs[ire] = e * t * cr;
        phd[ire] = e * n * t * cr;
        if (m >= 1) {
            phs[ire + 1] = -e * t * ci;
            phd[ire + 1] = -e * n * t * ci;
        }
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) deriv_all(phs, grad + d * K, L, d);
    __syncthreads();
    double* ch = A.chan + (size_t)s * K * nch;
    for (int q = threadIdx.x; q < K; q += blockDim.x) {
        ch[(size_t)q * nch + 0] = phs[q];
        for (int d = 0; d < 3; ++d) ch[(size_t)q * nch + 1 + d] = grad[d * K + q];
        ch[(size_t)q * nch + 4] = phd[q];
        ch[(size_t)q * nch + 5] = 0.0;
    }
}

// near_prep: one CTA per source sphere that has close partners.
// kind: 0 = S velocity, 1 = D velocity, 2 = S traction.
__global__ void near_prep_kernel(NearArgs A, int kind) {
    const int s = blockIdx.x;
    if (A.near_ptr[s + 1] == A.near_ptr[s]) return;
    const int p = A.p, P1 = p + 1, L = A.L, K = sh_count(L), nch = A.nch;
    extern __shared__ double sm[];
    double* base = sm;            // [5][K]  Pa, Pb, Pc, Pd, Pe
    double* grad = base + 5 * K;  // [4][3][K] grad of Pa, Pb, Pc, Pd
    double* tmp = grad + 12 * K;  // [K]
    const double* cf = A.coef ? A.coef + (size_t)s * 3 * P1 * P1 * 2 : nullptr;
    const float* cff = A.coef ? nullptr : A.coeff + (size_t)s * 3 * P1 * P1 * 2;
    for (int q = threadIdx.x; q < 5 * K; q += blockDim.x) base[q] = 0.0;
    __syncthreads();
    for (int q = threadIdx.x; q < P1 * P1; q += blockDim.x) {
        int n = q / P1, m = q - n * P1;
        if (m > n) continue;
        const double dn = (double)n;
        double sV, sW, cW, sX;
        if (kind == 1) {
            sV = (2 * dn * dn + 4 * dn + 3) / ((2 * dn + 1) * (2 * dn + 3));
            sW = 2 * (dn + 1) * (dn - 1) / ((2 * dn + 1) * (2 * dn - 1));
            cW = 2 * dn * (dn - 1) / (4 * dn + 2);
            sX = (dn - 1) / (2 * dn + 1);
        } else {
            sV = dn / ((2 * dn + 1) * (2 * dn + 3));
            sW = (dn + 1) / ((2 * dn + 1) * (2 * dn - 1));
            cW = dn / (4 * dn + 2);
            sX = 1.0 / (2 * dn + 1);
        }
        int o = n * P1 + m;
        auto co = [&](int i) { return cf ? cf[i] : (double)cff[i]; };
        double Vr = co(2 * o), Vi = co(2 * o + 1);
        double Wr = co(2 * (P1 * P1 + o)), Wi = co(2 * (P1 * P1 + o) + 1);
        double Xr = co(2 * (2 * P1 * P1 + o)), Xi = co(2 * (2 * P1 * P1 + o) + 1);
        if (n == 0) { Wr = Wi = Xr = Xi = 0.0; }
        double fr[5], fi[5];
        fr[0] = sV * Vr + cW * Wr; fi[0] = sV * Vi + cW * Wi;
        fr[1] = (sW - cW) * Wr;    fi[1] = (sW - cW) * Wi;
        fr[2] = (2 * dn + 1) * sW * Wr; fi[2] = (2 * dn + 1) * sW * Wi;
        fr[3] = sX * Xr;           fi[3] = sX * Xi;
        fr[4] = dn * Wr;           fi[4] = dn * Wi;
        double e = (m == 0 ? 1.0 : 2.0) * ynorm(n, m);
        int ire = sh_index(L, n, m, 0);
        for (int h = 0; h < 5; ++h) {
            base[h * K + ire] = e * fr[h];
            if (m >= 1) base[h * K + ire + 1] = -e * fi[h];
        }
    }
    __syncthreads();
    // gradients of Pa, Pb, Pc, Pd
    for (int h = 0; h < 4; ++h)
        for (int d = 0; d < 3; ++d) deriv_all(base + h * K, grad + (h * 3 + d) * K, L, d);
    __syncthreads();
    double* ch = A.chan + (size_t)s * K * nch;
    auto put = [&](int channel, const double* v) {
        for (int q = threadIdx.x; q < K; q += blockDim.x) ch[(size_t)q * nch + channel] = v[q];
    };
    if (kind < 2) {
        // [grad Pa (3), grad Pb (3), Pc, grad Pd (3)]
        for (int d = 0; d < 3; ++d) put(d, grad + (0 * 3 + d) * K);
        for (int d = 0; d < 3; ++d) put(3 + d, grad + (1 * 3 + d) * K);
        put(6, base + 2 * K);
        for (int d = 0; d < 3; ++d) put(7 + d, grad + (3 * 3 + d) * K);
    } else {
        // [hess Pa (6), grad Pb (3), hess Pb (6), Pc, grad Pc (3), hess Pd (6), Pe]
        const int hd0[6] = {0, 0, 0, 1, 1, 2}, hd1[6] = {0, 1, 2, 1, 2, 2};
        const int hset[3] = {0, 1, 3}, hch[3] = {0, 9, 19};
        for (int hs = 0; hs < 3; ++hs) {
            for (int e = 0; e < 6; ++e) {
                __syncthreads();
                deriv_all(grad + (hset[hs] * 3 + hd0[e]) * K, tmp, L, hd1[e]);
                __syncthreads();
                put(hch[hs] + e, tmp);
            }
        }
        for (int d = 0; d < 3; ++d) put(6 + d, grad + (1 * 3 + d) * K);
        put(15, base + 2 * K);
        for (int d = 0; d < 3; ++d) put(16 + d, grad + (2 * 3 + d) * K);
        put(25, base + 4 * K);
    }
    if (A.chanf) {
        __syncthreads();
        float* chf = A.chanf + (size_t)s * K * A.nchf;
        for (int q = threadIdx.x; q < K * A.nchf; q += blockDim.x) {
            int row = q / A.nchf, col = q - row * A.nchf;
            chf[q] = col < nch ? (float)ch[(size_t)row * nch + col] : 0.f;
        }
    }
}

// near_eval: CTA = (target sphere, chunk of its nodes); loops over the target's
// close source spheres, stages each source's channels in shared memory.
template <typename T, int NCH, int KIND>
__global__ void __launch_bounds__(128) near_eval_kernel(NearArgs A) {
    constexpr int NCHS = (sizeof(T) == 4) ? ((NCH + 3) / 4) * 4 : NCH;  // staged row width
    const int ti = blockIdx.x / A.chunks, chunk = blockIdx.x - ti * A.chunks;
    const int L = A.L, K = sh_count(L);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sch = reinterpret_cast<T*>(smraw);                 // [K][NCHS]
    T* rec = sch + (size_t)K * NCHS;                       // [2][K] recurrence factors (Re rows)
    // recurrence factors a1 = (2n-1)/(n-m), a2 = (n+m-1)/(n-m), indexed by the Re entry
    for (int m = 0; m <= L; ++m)
        for (int n = m + threadIdx.x; n <= L; n += blockDim.x) {
            int q = sh_index(L, n, m, 0);
            rec[q] = (n > m) ? (T)((2.0 * n - 1.0) / (n - m)) : (T)0;
            rec[K + q] = (n > m) ? (T)((n + m - 1.0) / (n - m)) : (T)0;
        }
    const int q = chunk * blockDim.x + threadIdx.x;
    const bool valid = q < A.npn;
    const long long node = (long long)ti * A.npn + (valid ? q : 0);
    const double X0 = A.x64[4 * node], Y0 = A.x64[4 * node + 1], Z0 = A.x64[4 * node + 2];
    const double nxv = A.nrm64[4 * node], nyv = A.nrm64[4 * node + 1], nzv = A.nrm64[4 * node + 2];
    double res[3] = {0.0, 0.0, 0.0};
    for (int e = A.near_ptr[ti]; e < A.near_ptr[ti + 1]; ++e) {
        const int k = A.near_idx[e];
        __syncthreads();
        if (sizeof(T) == 4) {
            const float4* src = reinterpret_cast<const float4*>(A.chanf + (size_t)k * K * NCHS);
            float4* dst = reinterpret_cast<float4*>(sch);
            for (int i = threadIdx.x; i < K * NCHS / 4; i += blockDim.x) dst[i] = src[i];
        } else {
            const double2* src = reinterpret_cast<const double2*>(A.chan + (size_t)k * K * NCH);
            double2* dst = reinterpret_cast<double2*>(sch);
            for (int i = threadIdx.x; i < K * NCH / 2; i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const double ak = A.radius[k];
        const double ia = 1.0 / ak;
        const T x = (T)((X0 - A.c[3 * k]) * ia), y = (T)((Y0 - A.c[3 * k + 1]) * ia), z = (T)((Z0 - A.c[3 * k + 2]) * ia);
        const T r2 = x * x + y * y + z * z;
        const T ir2 = (T)1 / r2;
        T acc[NCH];
#pragma unroll
        for (int h = 0; h < NCH; ++h) acc[h] = (T)0;
        // diagonal J_mm = (2m-1)!! (x + i y)^m / r^{2m+1}
        T dr = (T)1 / sqrt(r2), di = (T)0;
        for (int m = 0; m <= L; ++m) {
            if (m > 0) {
                T f = (T)(2 * m - 1) * ir2;
                T nr = (x * dr - y * di) * f;
                T ni = (x * di + y * dr) * f;
                dr = nr;
                di = ni;
            }
            T pr = (T)0, pi = (T)0;       // J_{n-2,m}
            T cr = dr, ci = di;           // J_{n-1,m} -> current
            int qre = sh_index(L, m, m, 0);
            const int step = (m == 0) ? 1 : 2;
            for (int n = m; n <= L; ++n) {
                if (n > m) {
                    T a1 = rec[qre] * z * ir2, a2 = rec[K + qre] * ir2;
                    T nr = a1 * cr - a2 * pr;
                    T ni = a1 * ci - a2 * pi;
                    pr = cr; pi = ci;
                    cr = nr; ci = ni;
                }
                const T* row = sch + (size_t)qre * NCHS;
#pragma unroll
                for (int h = 0; h < NCH; ++h) acc[h] = fma(row[h], cr, acc[h]);
                if (m > 0) {
                    const T* rowi = row + NCHS;
#pragma unroll
                    for (int h = 0; h < NCH; ++h) acc[h] = fma(rowi[h], ci, acc[h]);
                }
                qre += step;
            }
        }
        double xd = (double)x, yd = (double)y, zd = (double)z, rr = xd * xd + yd * yd + zd * zd;
        if (KIND == 3) {
            // Laplace value (S^L times the source radius, or D^L) or flux n . grad S^L
            // (grad in units of the source radius: the radius cancels)
            if (A.sel == 0) res[0] += ak * (double)acc[0];
            else if (A.sel == 1) res[0] += (double)acc[4];
            else res[0] += nxv * (double)acc[1] + nyv * (double)acc[2] + nzv * (double)acc[3];
        } else if (KIND == 4) {
            res[0] += (double)acc[1];
            res[1] += (double)acc[2];
            res[2] += (double)acc[3];
        } else if (KIND < 2) {
            // u = grad Pa + r^2 grad Pb + x Pc + x cross grad Pd
            double ga[3] = {acc[0], acc[1], acc[2]}, gb[3] = {acc[3], acc[4], acc[5]}, gd[3] = {acc[7], acc[8], acc[9]};
            double pc = acc[6];
            double u0 = ga[0] + rr * gb[0] + xd * pc + (yd * gd[2] - zd * gd[1]);
            double u1 = ga[1] + rr * gb[1] + yd * pc + (zd * gd[0] - xd * gd[2]);
            double u2 = ga[2] + rr * gb[2] + zd * pc + (xd * gd[1] - yd * gd[0]);
            double sc = (KIND == 0) ? ak : 1.0;
            res[0] += sc * u0; res[1] += sc * u1; res[2] += sc * u2;
        } else {
            // channels: Ha(0..5) gb(6..8) Hb(9..14) Pc(15) gc(16..18) Hd(19..24) Pe(25)
            auto hmul = [&](int o, double& a0, double& a1, double& a2) {
                double hxx = acc[o], hxy = acc[o + 1], hxz = acc[o + 2], hyy = acc[o + 3], hyz = acc[o + 4], hzz = acc[o + 5];
                a0 = hxx * nxv + hxy * nyv + hxz * nzv;
                a1 = hxy * nxv + hyy * nyv + hyz * nzv;
                a2 = hxz * nxv + hyz * nyv + hzz * nzv;
            };
            double han[3], hbn[3], hdn[3];
            hmul(0, han[0], han[1], han[2]);
            hmul(9, hbn[0], hbn[1], hbn[2]);
            hmul(19, hdn[0], hdn[1], hdn[2]);
            double gb[3] = {acc[6], acc[7], acc[8]}, gc[3] = {acc[16], acc[17], acc[18]};
            double pc = acc[15], pe = acc[25];
            double xv[3] = {xd, yd, zd}, nv[3] = {nxv, nyv, nzv};
            double xn = xd * nxv + yd * nyv + zd * nzv;
            double gbn = gb[0] * nxv + gb[1] * nyv + gb[2] * nzv;
            double gcn = gc[0] * nxv + gc[1] * nyv + gc[2] * nzv;
            // n cross x
            double nx_[3] = {nyv * zd - nzv * yd, nzv * xd - nxv * zd, nxv * yd - nyv * xd};
            double hd_nx[3];
            {
                int o = 19;
                double hxx = acc[o], hxy = acc[o + 1], hxz = acc[o + 2], hyy = acc[o + 3], hyz = acc[o + 4], hzz = acc[o + 5];
                hd_nx[0] = hxx * nx_[0] + hxy * nx_[1] + hxz * nx_[2];
                hd_nx[1] = hxy * nx_[0] + hyy * nx_[1] + hyz * nx_[2];
                hd_nx[2] = hxz * nx_[0] + hyz * nx_[1] + hzz * nx_[2];
            }
            double xc[3] = {yd * hdn[2] - zd * hdn[1], zd * hdn[0] - xd * hdn[2], xd * hdn[1] - yd * hdn[0]};
            for (int d = 0; d < 3; ++d) {
                res[d] += 2.0 * han[d] + 2.0 * xn * gb[d] + 2.0 * gbn * xv[d] + 2.0 * rr * hbn[d] + 2.0 * pc * nv[d] +
                          gcn * xv[d] + xn * gc[d] + xc[d] + hd_nx[d] - pe * nv[d];
            }
        }
    }
    if (valid) {
        double* o = A.out + node * 3;
        o[0] += res[0];
        o[1] += res[1];
        o[2] += res[2];
    }
}


template <typename T, int NCH, int KIND>
static cudaError_t run_eval(sbie_ctx* c, const NearArgs& A) {
    constexpr int NCHS = (sizeof(T) == 4) ? ((NCH + 3) / 4) * 4 : NCH;
    int K = sh_count(A.L);
    size_t sm = sizeof(T) * ((size_t)K * NCHS + 2 * K);
    cudaError_t e = cudaFuncSetAttribute(near_eval_kernel<T, NCH, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    near_eval_kernel<T, NCH, KIND><<<c->n * A.chunks, A.threads, sm, c->stream>>>(A); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_near_prep_pairs(sbie_ctx* c, int kind, int count, const double* coef, const float* coeff,
                                   const int* iota, double* chan, float* chanf) {
    NearArgs A{};
    A.n = count; A.p = c->p; A.npn = c->npn;
    A.L = (kind == 2) ? c->p + 2 : c->p + 1;
    A.nch = (kind == 2) ? kTracChannels : kVelChannels;
    A.nchf = chanf ? (A.nch + 3) / 4 * 4 : 0;
    A.coef = coef; A.coeff = coeff; A.near_ptr = iota; A.chan = chan; A.chanf = chanf;
    const int K = sh_count(A.L);
    const size_t sm = sizeof(double) * (size_t)(5 * K + 12 * K + K);
    cudaError_t e = cudaFuncSetAttribute(near_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    near_prep_kernel<<<count, 256, sm, c->stream>>>(A, kind); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_near_laplace(sbie_ctx* c, int mode, double* out) {
    if (c->n_near == 0) return cudaSuccess;
    NearArgs A{};
    A.n = c->n; A.p = c->p; A.npn = c->npn;
    A.L = c->p + 1;
    A.nch = kLapChannels;
    A.nchf = ((A.nch + 3) / 4) * 4;
    A.sel = mode == kLapSL ? 0 : (mode == kLapDL ? 1 : 2);
    A.threads = 128;
    while (A.threads > 32 && (long long)c->n * ((c->npn + A.threads - 1) / A.threads) < 2LL * c->sm_count)
        A.threads /= 2;
    A.chunks = (c->npn + A.threads - 1) / A.threads;
    A.coef = c->d_lcoef; A.radius = c->d_a; A.c = c->d_c; A.x64 = c->d_x; A.nrm64 = c->d_nrm64;
    A.near_ptr = c->d_near_ptr; A.near_idx = c->d_near_idx;
    A.chan = c->d_chan; A.chanf = nullptr; A.out = out;
    const int K = sh_count(A.L);
    const size_t sm = sizeof(double) * (size_t)(5 * K);
    cudaError_t e = cudaFuncSetAttribute(near_prep_laplace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    near_prep_laplace_kernel<<<c->n, 256, sm, c->stream>>>(A); ++c->n_launch;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mode == kLapGrad) return run_eval<double, kLapChannels, 4>(c, A);
    return run_eval<double, kLapChannels, 3>(c, A);
}

cudaError_t launch_near(sbie_ctx* c, Kern op, bool f32, double* out) {
    if (c->n_near == 0) return cudaSuccess;
    NearArgs A{};
    A.n = c->n; A.p = c->p; A.npn = c->npn;
    int kind = (op == Kern::S) ? 0 : (op == Kern::D ? 1 : 2);
    A.L = (kind == 2) ? c->p + 2 : c->p + 1;
    A.nch = (kind == 2) ? kTracChannels : kVelChannels;
    A.nchf = ((A.nch + 3) / 4) * 4;
    // targets per CTA: 128, or fewer when a small suspension would leave most
    // SMs idle (the source channels are then staged by more CTAs)
    A.threads = 128;
    while (A.threads > 32 && (long long)c->n * ((c->npn + A.threads - 1) / A.threads) < 2LL * c->sm_count)
        A.threads /= 2;
    A.chunks = (c->npn + A.threads - 1) / A.threads;
    A.coef = c->d_coef; A.radius = c->d_a; A.c = c->d_c; A.x64 = c->d_x; A.nrm64 = c->d_nrm64;
    A.near_ptr = c->d_near_ptr; A.near_idx = c->d_near_idx;
    A.chan = c->d_chan; A.chanf = f32 ? c->d_chanf : nullptr; A.out = out;
    int K = sh_count(A.L);
    size_t sm = sizeof(double) * (size_t)(5 * K + 12 * K + K);
    cudaError_t e = cudaFuncSetAttribute(near_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    near_prep_kernel<<<c->n, 256, sm, c->stream>>>(A, kind); ++c->n_launch;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (f32) {
        if (kind == 0) return run_eval<float, kVelChannels, 0>(c, A);
        if (kind == 1) return run_eval<float, kVelChannels, 1>(c, A);
        return run_eval<float, kTracChannels, 2>(c, A);
    }
    if (kind == 0) return run_eval<double, kVelChannels, 0>(c, A);
    if (kind == 1) return run_eval<double, kVelChannels, 1>(c, A);
    return run_eval<double, kTracChannels, 2>(c, A);
}

}  // namespace sbie
