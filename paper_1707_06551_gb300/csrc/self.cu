// Self interaction of each sphere (Sec. 4.1, Eqs. 4.6-4.7): VSH analysis of the
// density (Sec. 2.1), multiplication by the operator's signature (Theorem 2,
// Eq. 3.12) and synthesis on the same grid (Eqs. 2.15-2.17).
//
// One CTA per sphere, everything in shared memory, FP64.  The transform is a
// direct DFT in phi (2p+2 points) followed by a Gauss-Legendre contraction in
// theta; the analysis is the exact projection onto V, W, X (for a band-limited
// density the grid integrates every product exactly).  The coefficients are
// also written to global memory for the close-pair kernels.
#include "common.h"

namespace sbie {

struct SelfArgs {
    int p, nlat, nlon, npn;
    TabLayout tl;
    const double* tab;
    const double* dens;   // [N][3]
    double* out;          // [N][3]
    double* coef;         // [n][3][p+1][p+1][2] or nullptr
    const double* radius; // [n]
    int op;               // -1 = analysis only, else Kern
    int accumulate;
};

__device__ __forceinline__ void signature(int op, int n, double a, double& lv, double& lw, double& lx) {
    double tn1 = 2.0 * n + 1.0;
    if (op == kOpPrecHigh) {
        if (n > 4) {
            lv = (tn1 * (2.0 * n + 3.0)) / (2.0 * n * n + 4.0 * n + 3.0);
            lw = (tn1 * (2.0 * n - 1.0)) / (2.0 * (n - 1.0) * (n + 1.0));
            lx = tn1 / (n - 1.0);
        } else {
            lv = lw = lx = 0.0;
        }
        lv -= 2.0;
        lw -= 2.0;
        lx -= 2.0;
        return;
    }
    if (op == (int)Kern::S) {
        lv = n / (tn1 * (2.0 * n + 3.0));
        lw = (n + 1.0) / (tn1 * (2.0 * n - 1.0));
        lx = 1.0 / tn1;
        lv *= a;
        lw *= a;
        lx *= a;
    } else {
        // principal value (D+ + D-)/2 = (K+ + K-)/2
        lv = 3.0 / (2.0 * tn1 * (2.0 * n + 3.0));
        lw = -3.0 / (2.0 * tn1 * (2.0 * n - 1.0));
        lx = -3.0 / (2.0 * tn1);
    }
}

__global__ void self_kernel(SelfArgs A) {
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

    extern __shared__ double sm[];
    double* f = sm;                           // [3][npn]
    double* Fh = f + 3 * npn;                 // [3][nlat][P1][2]
    double* cf = Fh + 3 * nlat * P1 * 2;      // [3][P1][P1][2]
    const int tid = threadIdx.x, bd = blockDim.x;
    const size_t base = (size_t)s * npn;

    // 1. spherical components (f_r, f_theta, f_phi) at every node
    for (int q = tid; q < npn; q += bd) {
        int j = q / nlon, k = q - j * nlon;
        const double* d = A.dens + (base + q) * 3;
        double fx = d[0], fy = d[1], fz = d[2];
        double c = ct[j], sn = st[j], cp = cph[k], sp = sph[k];
        f[q] = fx * sn * cp + fy * sn * sp + fz * c;
        f[npn + q] = fx * c * cp + fy * c * sp - fz * sn;
        f[2 * npn + q] = -fx * sp + fy * cp;
    }
    __syncthreads();
    // 2. DFT in phi: Fh[c][j][m] = sum_k f e^{-i m phi_k}
    for (int q = tid; q < 3 * nlat * P1; q += bd) {
        int c = q / (nlat * P1), r = q - c * nlat * P1, j = r / P1, m = r - j * P1;
        const double* row = f + c * npn + j * nlon;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < nlon; ++k) {
            double v = row[k];
            re = fma(v, cmk[m * nlon + k], re);
            im = fma(-v, smk[m * nlon + k], im);
        }
        Fh[2 * q] = re;
        Fh[2 * q + 1] = im;
    }
    __syncthreads();
    // 3. Legendre contraction -> (phi^Y, phi^G, phi^X) -> (V, W, X) coefficients
    for (int q = tid; q < P1 * P1; q += bd) {
        int m = q / P1, n = q - m * P1;
        double vr = 0, vi = 0, wr = 0, wi = 0, xr = 0, xi = 0;
        if (m <= n) {
            double yr = 0, yi = 0, gr = 0, gi = 0, hr = 0, hi = 0;
            for (int j = 0; j < nlat; ++j) {
                int o = (m * P1 + n) * nlat + j;
                double w = wq[j], P = Pt[o] * w, dP = dPt[o] * w, mS = mSt[o] * w;
                const double* Fr = Fh + 2 * ((0 * nlat + j) * P1 + m);
                const double* Ft = Fh + 2 * ((1 * nlat + j) * P1 + m);
                const double* Fp = Fh + 2 * ((2 * nlat + j) * P1 + m);
                yr = fma(P, Fr[0], yr);
                yi = fma(P, Fr[1], yi);
                // G: dP F_theta - i mS F_phi ; X: i mS F_theta + dP F_phi
                gr += dP * Ft[0] + mS * Fp[1];
                gi += dP * Ft[1] - mS * Fp[0];
                hr += -mS * Ft[1] + dP * Fp[0];
                hi += mS * Ft[0] + dP * Fp[1];
            }
            if (n == 0) {
                vr = -yr;
                vi = -yi;
            } else {
                double inn = 1.0 / (n * (n + 1.0));
                gr *= inn; gi *= inn; hr *= inn; hi *= inn;
                double t = 1.0 / (2.0 * n + 1.0);
                vr = (n * gr - yr) * t;
                vi = (n * gi - yi) * t;
                wr = ((n + 1.0) * gr + yr) * t;
                wi = ((n + 1.0) * gi + yi) * t;
                xr = hr;
                xi = hi;
            }
            if (m == 0) { vi = 0; wi = 0; xi = 0; }
        }
        if (A.coef) {
            double* cg = A.coef + (size_t)s * 3 * P1 * P1 * 2;
            int o = n * P1 + m;
            cg[2 * o] = vr; cg[2 * o + 1] = vi;
            cg[2 * (P1 * P1 + o)] = wr; cg[2 * (P1 * P1 + o) + 1] = wi;
            cg[2 * (2 * P1 * P1 + o)] = xr; cg[2 * (2 * P1 * P1 + o) + 1] = xi;
        }
        if (A.op >= 0) {
            double lv, lw, lx;
            signature(A.op, n, A.radius[s], lv, lw, lx);
            vr *= lv; vi *= lv; wr *= lw; wi *= lw; xr *= lx; xi *= lx;
            // back to (Y, G, X): phi^Y = -(n+1) V + n W, phi^G = V + W
            int o = (n * P1 + m) * 2;
            cf[o] = -(n + 1.0) * vr + n * wr;
            cf[o + 1] = -(n + 1.0) * vi + n * wi;
            cf[2 * P1 * P1 + o] = vr + wr;
            cf[2 * P1 * P1 + o + 1] = vi + wi;
            cf[4 * P1 * P1 + o] = xr;
            cf[4 * P1 * P1 + o + 1] = xi;
        }
    }
    if (A.op < 0) return;
    __syncthreads();
    // 4. inverse Legendre: A_c(j, m), stored in Fh
    for (int q = tid; q < 3 * nlat * P1; q += bd) {
        int c = q / (nlat * P1), r = q - c * nlat * P1, j = r / P1, m = r - j * P1;
        double ar = 0, ai = 0;
        for (int n = m; n <= p; ++n) {
            int o = (m * P1 + n) * nlat + j;
            int oc = (n * P1 + m) * 2;
            double Yr = cf[oc], Yi = cf[oc + 1];
            double Gr = cf[2 * P1 * P1 + oc], Gi = cf[2 * P1 * P1 + oc + 1];
            double Xr = cf[4 * P1 * P1 + oc], Xi = cf[4 * P1 * P1 + oc + 1];
            if (c == 0) {
                double P = Pt[o];
                ar = fma(Yr, P, ar);
                ai = fma(Yi, P, ai);
            } else if (c == 1) {  // G dP - i X mS
                double dP = dPt[o], mS = mSt[o];
                ar += Gr * dP + Xi * mS;
                ai += Gi * dP - Xr * mS;
            } else {              // i G mS + X dP
                double dP = dPt[o], mS = mSt[o];
                ar += -Gi * mS + Xr * dP;
                ai += Gr * mS + Xi * dP;
            }
        }
        Fh[2 * q] = ar;
        Fh[2 * q + 1] = ai;
    }
    __syncthreads();
    // 5. inverse DFT: f = Re A(0) + 2 Re sum_{m>=1} A(m) e^{i m phi_k}
    for (int q = tid; q < 3 * npn; q += bd) {
        int c = q / npn, r = q - c * npn, j = r / nlon, k = r - j * nlon;
        const double* a = Fh + 2 * ((c * nlat + j) * P1);
        double v = 0.0;
        for (int m = 1; m <= p; ++m) {
            v = fma(a[2 * m], cmk[m * nlon + k], v);
            v = fma(-a[2 * m + 1], smk[m * nlon + k], v);
        }
        f[q] = a[0] + 2.0 * v;
    }
    __syncthreads();
    // 6. back to Cartesian; write or accumulate
    for (int q = tid; q < npn; q += bd) {
        int j = q / nlon, k = q - j * nlon;
        double c = ct[j], sn = st[j], cp = cph[k], sp = sph[k];
        double fr = f[q], ft = f[npn + q], fp = f[2 * npn + q];
        double ox = fr * sn * cp + ft * c * cp - fp * sp;
        double oy = fr * sn * sp + ft * c * sp + fp * cp;
        double oz = fr * c - ft * sn;
        double* o = A.out + (base + q) * 3;
        if (A.accumulate) {
            o[0] += ox; o[1] += oy; o[2] += oz;
        } else {
            o[0] = ox; o[1] = oy; o[2] = oz;
        }
    }
}

static size_t self_smem(int p) {
    int P1 = p + 1, nlat = p + 1, npn = (p + 1) * (2 * p + 2);
    return sizeof(double) * (size_t)(3 * npn + 3 * nlat * P1 * 2 + 3 * P1 * P1 * 2);
}

static cudaError_t run_self(sbie_ctx* c, int op, const double* dens, double* out, bool accumulate, bool write_coef) {
    SelfArgs A;
    A.p = c->p; A.nlat = c->nlat; A.nlon = c->nlon; A.npn = c->npn;
    A.tl = c->tl; A.tab = c->d_tab; A.dens = dens; A.out = out;
    A.coef = write_coef ? c->d_coef : nullptr;
    A.radius = c->d_a; A.op = op; A.accumulate = accumulate ? 1 : 0;
    size_t sm = self_smem(c->p);
    // The shared-memory opt-in is a per-device attribute of the kernel: set it
    // on every launch that needs more than the 48 KB default (p >= 17), so the
    // device current at this launch has it whichever device ran first.  One
    // fixed value for all orders, so that concurrent launches of different
    // orders never lower it under one another.
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(self_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    self_kernel<<<c->n, 256, sm, c->stream>>>(A); ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_self(sbie_ctx* c, Kern op, const double* dens, double* out, bool accumulate, bool write_coef) {
    return run_self(c, (int)op, dens, out, accumulate, write_coef);
}

cudaError_t launch_self_precond(sbie_ctx* c, const double* v, double* out) {
    return run_self(c, kOpPrecHigh, v, out, false, true);
}

cudaError_t launch_self_analysis(sbie_ctx* c, const double* dens) {
    return run_self(c, -1, dens, nullptr, false, true);
}

cudaError_t launch_self_probe(sbie_ctx* c, int op, int count, const double* dens, double* out, const double* radius,
                              double* coef) {
    SelfArgs A;
    A.p = c->p; A.nlat = c->nlat; A.nlon = c->nlon; A.npn = c->npn;
    A.tl = c->tl; A.tab = c->d_tab; A.dens = dens; A.out = out;
    A.coef = coef;
    A.radius = radius; A.op = op; A.accumulate = 0;
    const size_t sm = self_smem(c->p);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(self_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    self_kernel<<<count, 256, sm, c->stream>>>(A); ++c->n_launch;
    return cudaGetLastError();
}


}  // namespace sbie
