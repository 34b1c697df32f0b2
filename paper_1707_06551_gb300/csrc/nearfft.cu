// Close pairs by the rotated, FFT-accelerated scheme of Sec. 4.2 (Fig. 2).
//
// For each directed close pair (source k, target i), in the frame x' = Q x whose
// pole points from c_k to c_i (Q^T = R_z(a) R_y(b), (sin b cos a, sin b sin a,
// cos b) the unit vector from c_k to c_i):
//   (1) the source's VSH coefficients are rotated to that frame (degree by
//       degree: f -> f o Q^T = Z(a), then the 90-degree x rotation Mm, Z(b),
//       Mp, with Z(t) the phase e^{i m t} of order m -- R_y(b) = R_x(-90) R_z(b)
//       R_x(90); V, W and X rotate as Y);
//   (2) the target sphere's grid, placed about the target centre in that frame,
//       lies on p+1 discs about the pole (constant r and theta, equispaced
//       phi): the source's exterior expansion -- the solid-harmonic channels of
//       near.cu built from the rotated coefficients -- is summed over n for each
//       (disc, m) and then over m for each phi (a discrete Fourier sum), and the
//       channels combined into the velocity (S, D) or the traction (K, with the
//       target's normals) at every rotated node;
//   (3) those samples, a vector field on the target sphere in the rotated
//       frame, are analysed on its grid (forward VSH transform), the
//       coefficients rotated back (Mm, Z(-b), Mp, Z(-a)), and the blocks of all
//       close sources of a target sphere summed in a fixed order and
//       synthesised at its nodes.
// Stage (3) projects the close-pair field onto degree <= p on the target
// sphere, as the paper's algorithm does.  Per pair the work is O(p^3) (one
// CTA per pair), against O(p^4) for the direct evaluation of near.cu.
//
// Arithmetic T: FP64 for the FP64 and FP64-accurate operators; FP32 for the
// FP32 operator of the mixed path (the channels are built in FP64 from the
// FP32 rotated coefficients and read in FP32, as the direct scheme's are).
#include <algorithm>

#include "common.h"

namespace sbie {

namespace {

template <typename T>
struct FftArgs {
    int p, P1, L, K, nchs, npn, nlat, nlon, n_near, G;  // nchs: channel row stride; G: discs evaluated together
    TabLayout tl;
    const T* tab;
    const T* rotp;        // f -> f o R_x(+90) per degree
    const T* rotm;        // f -> f o R_x(-90)
    const double* geo;    // [n_near][8]: cos a, sin a, cos b, sin b, d / a_s, a_t / a_s, a_s, unused
    const double* coef;   // [n][3][P1 (n)][P1 (m)][2] source coefficients
    const int* near_ptr;  // CSR by target sphere
    const int* near_idx;  // source sphere of each entry
    T* pcoef;             // [n_near][3][P1][P1][2] rotated source coefficients
    const T* chan;        // [n_near][K][nchs]
    T* blk;               // [n_near][3][P1][P1][2] target-side coefficient blocks
    double* out;          // [N][3]
};

__device__ __forceinline__ int rot_off(int n) { return n * (2 * n - 1) * (2 * n + 1) / 3; }

// degree n of the full-vector index r = n^2 + (m + n)
__device__ __forceinline__ int degree_of(int r) {
    int n = (int)sqrtf((float)r + 0.5f);
    while ((n + 1) * (n + 1) <= r) ++n;
    while (n * n > r) --n;
    return n;
}

// e^{i m t} from cos t, sin t by repeated multiplication
template <typename T>
__device__ __forceinline__ void phase_pow(T c, T s, int m, T& cm, T& sm) {
    cm = T(1);
    sm = T(0);
    for (int k = 0; k < m; ++k) {
        const T nc = cm * c - sm * s;
        sm = sm * c + cm * s;
        cm = nc;
    }
}

// Rotate 3 VSH coefficient sets (layout [3][P1 (n)][P1 (m)][2], m >= 0 of a real
// field) from `in` to `out` (both shared), `v`, `w` scratch of 3 * (p+1)^2
// complex each.  forward: f o Q^T; else f o Q.
template <typename T>
__device__ void rotate_vsh(const FftArgs<T>& A, const T* in, T* out, T* v, T* w, T ca, T sa, T cb, T sb,
                           bool forward) {
    const int P1 = A.P1, S = P1 * P1;  // full vectors: index n^2 + (m + n)
    const int tid = threadIdx.x, bd = blockDim.x;
    // full complex vectors, with the first phase applied when forward: Z(a)
    for (int q = tid; q < 3 * S; q += bd) {
        const int t = q / S, r = q - t * S;
        const int n = degree_of(r);
        const int m = r - n * n - n;
        const int am = m < 0 ? -m : m;
        const T* c = in + 2 * ((t * P1 + n) * P1 + am);
        T re = c[0], im = m < 0 ? -c[1] : c[1];
        if (forward) {  // e^{i m a}
            T cm, sm;
            phase_pow(ca, sa, am, cm, sm);
            if (m < 0) sm = -sm;
            const T nr = re * cm - im * sm;
            im = re * sm + im * cm;
            re = nr;
        }
        v[2 * q] = re;
        v[2 * q + 1] = im;
    }
    __syncthreads();
    // w = Mm v, then the phase e^{+- i m b}
    for (int q = tid; q < 3 * S; q += bd) {
        const int t = q / S, r = q - t * S;
        const int n = degree_of(r);
        const int mr = r - n * n - n, wdt = 2 * n + 1;
        const T* M = A.rotm + 2 * ((size_t)rot_off(n) + (size_t)(mr + n) * wdt);
        const T* x = v + 2 * (t * S + n * n);
        T re = T(0), im = T(0);
        for (int c = 0; c < wdt; ++c) {
            re += M[2 * c] * x[2 * c] - M[2 * c + 1] * x[2 * c + 1];
            im += M[2 * c] * x[2 * c + 1] + M[2 * c + 1] * x[2 * c];
        }
        T cm, sm;
        phase_pow(cb, sb, mr < 0 ? -mr : mr, cm, sm);
        if ((mr < 0) == forward) sm = -sm;  // forward: e^{i m b}; back: e^{-i m b}
        w[2 * q] = re * cm - im * sm;
        w[2 * q + 1] = re * sm + im * cm;
    }
    __syncthreads();
    // out = Mp w (m >= 0), then when going back the phase e^{-i m a}
    for (int q = tid; q < 3 * P1 * P1; q += bd) {
        const int t = q / (P1 * P1), r = q - t * P1 * P1, n = r / P1, m = r - n * P1;
        T re = T(0), im = T(0);
        if (m <= n) {
            const int wdt = 2 * n + 1;
            const T* M = A.rotp + 2 * ((size_t)rot_off(n) + (size_t)(m + n) * wdt);
            const T* x = w + 2 * (t * S + n * n);
            for (int c = 0; c < wdt; ++c) {
                re += M[2 * c] * x[2 * c] - M[2 * c + 1] * x[2 * c + 1];
                im += M[2 * c] * x[2 * c + 1] + M[2 * c + 1] * x[2 * c];
            }
            if (!forward) {
                T cm, sm;
                phase_pow(ca, sa, m, cm, sm);
                const T nr = re * cm + im * sm;  // times e^{-i m a}
                im = im * cm - re * sm;
                re = nr;
            }
            if (m == 0) im = T(0);
            if (t > 0 && n == 0) re = im = T(0);
        }
        out[2 * q] = re;
        out[2 * q + 1] = im;
    }
    __syncthreads();
}

// stage (1): one CTA per entry e of the close-pair lists
template <typename T>
__global__ void fft_rotate_kernel(FftArgs<T> A) {
    const int e = blockIdx.x;
    const int P1 = A.P1, S = P1 * P1;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* cin = reinterpret_cast<T*>(smraw);  // [3][P1][P1][2]
    T* cout = cin + 6 * S;
    T* v = cout + 6 * S;                   // [3][P1^2][2]
    T* w = v + 6 * S;
    const int k = A.near_idx[e];
    const double* src = A.coef + (size_t)k * 6 * S;
    for (int q = threadIdx.x; q < 6 * S; q += blockDim.x) cin[q] = (T)src[q];
    __syncthreads();
    const double* g = A.geo + 8 * (size_t)e;
    rotate_vsh(A, cin, cout, v, w, (T)g[0], (T)g[1], (T)g[2], (T)g[3], true);
    T* dst = A.pcoef + (size_t)e * 6 * S;
    for (int q = threadIdx.x; q < 6 * S; q += blockDim.x) dst[q] = cout[q];
}

// stages (2) and (3): one CTA per entry e; KIND 0 = S, 1 = D (velocity
// channels), 2 = traction of S.  The discs are evaluated G at a time so that
// every thread has a node.
template <typename T, int KIND>
__global__ void fft_eval_kernel(FftArgs<T> A) {
    constexpr int NCH = KIND == 2 ? kTracChannels : kVelChannels;
    const int e = blockIdx.x;
    const int P1 = A.P1, L = A.L, K = A.K, nchs = A.nchs, npn = A.npn, nlat = A.nlat, nlon = A.nlon, G = A.G;
    const TabLayout& tl = A.tl;
    const T* tab = A.tab;
    const T* ct = tab + tl.o_ct;
    const T* st = tab + tl.o_st;
    const T* wq = tab + tl.o_w;
    const T* cph = tab + tl.o_cph;
    const T* sph = tab + tl.o_sph;
    const T* cmk = tab + tl.o_cmk;
    const T* smk = tab + tl.o_smk;
    const T* Pt = tab + tl.o_P;
    const T* dPt = tab + tl.o_dP;
    const T* mSt = tab + tl.o_mS;
    const int S = P1 * P1;
    extern __shared__ __align__(16) unsigned char smraw[];
    // the pair's channels stay in global memory (read through L1): at p = 24
    // they alone would fill the shared memory
    const T* ch = A.chan + (size_t)e * K * nchs;  // [K][nchs]
    T* Ad = reinterpret_cast<T*>(smraw);          // [G][L+1][NCH][2] a group of discs
    T* U = Ad + (size_t)G * (L + 1) * NCH * 2;   // [3][npn] spherical components of the samples
    T* Fh = U + 3 * npn;                         // [3][nlat][P1][2]
    T* cu = Fh + 3 * nlat * P1 * 2;              // [3][P1][P1][2]
    T* cv = cu + 6 * S;                          // [3][P1][P1][2]
    T* v = cv + 6 * S;                           // rotation scratch [3][P1^2][2] x 2
    T* w = v + 6 * S;
    T* pc = w + 6 * S;                           // [nlon] cos, [nlon] sin of 2 pi q / nlon
    T* ps = pc + nlon;
    const int tid = threadIdx.x, bd = blockDim.x;
    const double* g = A.geo + 8 * (size_t)e;
    const T D = (T)g[4], rho = (T)g[5], scale = KIND == 0 ? (T)g[6] : T(1);  // S scales by the source radius
    for (int q = tid; q < nlon; q += bd) {
        pc[q] = cph[q];
        ps[q] = sph[q];
    }
    // (2) disc by disc, G discs at a time
    for (int j0 = 0; j0 < nlat; j0 += G) {
        const int gs = min(G, nlat - j0);
        __syncthreads();
        // A_hm = sum_n (ch_re - i ch_im)(n, m, h) P_n^m(t) / r^{n+1}, t and r of the disc
        for (int q = tid; q < gs * (L + 1) * NCH; q += bd) {
            const int jj = q / ((L + 1) * NCH), r = q - jj * (L + 1) * NCH, m = r / NCH, h = r - m * NCH;
            const int j = j0 + jj;
            const T zj = D + rho * ct[j], pj = rho * st[j];
            const T rj = sqrt(zj * zj + pj * pj), ir = T(1) / rj, tj = zj * ir, sj = pj * ir;
            T qmm = ir;  // (2m-1)!! s^m / r^{m+1}
            for (int k = 1; k <= m; ++k) qmm *= (T)(2 * k - 1) * sj * ir;
            T q0 = T(0), q1 = qmm, ar = T(0), ai = T(0);
            for (int n = m; n <= L; ++n) {
                T qn;
                if (n == m) {
                    qn = qmm;
                } else {
                    qn = ((T)(2 * n - 1) * tj * ir * q1 - (T)(n + m - 1) * ir * ir * q0) / (T)(n - m);
                    q0 = q1;
                    q1 = qn;
                }
                const int ire = sh_index(L, n, m, 0);
                ar = fma(ch[(size_t)ire * nchs + h], qn, ar);
                if (m >= 1) ai = fma(-ch[(size_t)(ire + 1) * nchs + h], qn, ai);
            }
            Ad[2 * q] = ar;
            Ad[2 * q + 1] = ai;
        }
        __syncthreads();
        // channel values at the group's nodes (Fourier sums over the orders),
        // combined into the velocity or traction
        for (int qq = tid; qq < gs * nlon; qq += bd) {
            const int jj = qq / nlon, k = qq - jj * nlon, j = j0 + jj;
            const T* Aj = Ad + (size_t)jj * (L + 1) * NCH * 2;
            T val[NCH];
#pragma unroll
            for (int h = 0; h < NCH; ++h) val[h] = T(0);
            int ph = 0;  // m k mod nlon
            for (int m = 0; m <= L; ++m) {
                const T c = pc[ph], s = ps[ph];
                ph += k;
                if (ph >= nlon) ph -= nlon;
                const T* a = Aj + 2 * m * NCH;
#pragma unroll
                for (int h = 0; h < NCH; ++h) val[h] = fma(a[2 * h], c, fma(-a[2 * h + 1], s, val[h]));
            }
            // point (source units) and target normal in the rotated frame
            const T dx = st[j] * pc[k], dy = st[j] * ps[k], dz = ct[j];
            const T xd = rho * dx, yd = rho * dy, zd = D + rho * dz;
            T u0, u1, u2;
            if (KIND < 2) {
                const T rr = xd * xd + yd * yd + zd * zd;
                u0 = val[0] + rr * val[3] + xd * val[6] + (yd * val[9] - zd * val[8]);
                u1 = val[1] + rr * val[4] + yd * val[6] + (zd * val[7] - xd * val[9]);
                u2 = val[2] + rr * val[5] + zd * val[6] + (xd * val[8] - yd * val[7]);
            } else {
                const T nxv = dx, nyv = dy, nzv = dz, rr = xd * xd + yd * yd + zd * zd;
                auto hm = [&](int o, T a0, T a1, T a2, T& r0, T& r1, T& r2) {
                    r0 = val[o] * a0 + val[o + 1] * a1 + val[o + 2] * a2;
                    r1 = val[o + 1] * a0 + val[o + 3] * a1 + val[o + 4] * a2;
                    r2 = val[o + 2] * a0 + val[o + 4] * a1 + val[o + 5] * a2;
                };
                T han[3], hbn[3], hdn[3], hdx[3];
                hm(0, nxv, nyv, nzv, han[0], han[1], han[2]);
                hm(9, nxv, nyv, nzv, hbn[0], hbn[1], hbn[2]);
                hm(19, nxv, nyv, nzv, hdn[0], hdn[1], hdn[2]);
                const T nx_[3] = {nyv * zd - nzv * yd, nzv * xd - nxv * zd, nxv * yd - nyv * xd};
                hm(19, nx_[0], nx_[1], nx_[2], hdx[0], hdx[1], hdx[2]);
                const T gb[3] = {val[6], val[7], val[8]}, gc[3] = {val[16], val[17], val[18]};
                const T pcv = val[15], pe = val[25];
                const T xv[3] = {xd, yd, zd}, nv[3] = {nxv, nyv, nzv};
                const T xn = xd * nxv + yd * nyv + zd * nzv;
                const T gbn = gb[0] * nxv + gb[1] * nyv + gb[2] * nzv;
                const T gcn = gc[0] * nxv + gc[1] * nyv + gc[2] * nzv;
                const T xc[3] = {yd * hdn[2] - zd * hdn[1], zd * hdn[0] - xd * hdn[2], xd * hdn[1] - yd * hdn[0]};
                T t3[3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    t3[d] = T(2) * han[d] + T(2) * xn * gb[d] + T(2) * gbn * xv[d] + T(2) * rr * hbn[d] +
                            T(2) * pcv * nv[d] + gcn * xv[d] + xn * gc[d] + xc[d] + hdx[d] - pe * nv[d];
                u0 = t3[0];
                u1 = t3[1];
                u2 = t3[2];
            }
            // spherical components about the target centre: (e_r, e_theta, e_phi) of the node
            const int q = j * nlon + k;
            const T c = ct[j], sn = st[j], cp = pc[k], sp = ps[k];
            U[q] = u0 * sn * cp + u1 * sn * sp + u2 * c;
            U[npn + q] = u0 * c * cp + u1 * c * sp - u2 * sn;
            U[2 * npn + q] = -u0 * sp + u1 * cp;
        }
    }
    __syncthreads();
    // (3) forward VSH transform on the target grid: DFT in phi, Legendre, (Y, G, X) -> (V, W, X)
    for (int q = tid; q < 3 * nlat * P1; q += bd) {
        const int c = q / (nlat * P1), r = q - c * nlat * P1, j = r / P1, m = r - j * P1;
        const T* row = U + c * npn + j * nlon;
        T re = T(0), im = T(0);
        for (int k = 0; k < nlon; ++k) {
            re = fma(row[k], cmk[m * nlon + k], re);
            im = fma(-row[k], smk[m * nlon + k], im);
        }
        Fh[2 * q] = re;
        Fh[2 * q + 1] = im;
    }
    __syncthreads();
    for (int q = tid; q < P1 * P1; q += bd) {
        const int n = q / P1, m = q - n * P1;
        T vr = T(0), vi = T(0), wr = T(0), wi = T(0), xr = T(0), xi = T(0);
        if (m <= n) {
            T yr = T(0), yi = T(0), gr = T(0), gi = T(0), hr = T(0), hi = T(0);
            for (int j = 0; j < nlat; ++j) {
                const int o = (m * P1 + n) * nlat + j;
                const T wj = wq[j], P = Pt[o] * wj, dP = dPt[o] * wj, mS = mSt[o] * wj;
                const T* Fr = Fh + 2 * ((0 * nlat + j) * P1 + m);
                const T* Ft = Fh + 2 * ((1 * nlat + j) * P1 + m);
                const T* Fp = Fh + 2 * ((2 * nlat + j) * P1 + m);
                yr = fma(P, Fr[0], yr);
                yi = fma(P, Fr[1], yi);
                gr += dP * Ft[0] + mS * Fp[1];
                gi += dP * Ft[1] - mS * Fp[0];
                hr += -mS * Ft[1] + dP * Fp[0];
                hi += mS * Ft[0] + dP * Fp[1];
            }
            if (n == 0) {
                vr = -yr;
                vi = -yi;
            } else {
                const T inn = T(1) / (T)(n * (n + 1)), t = T(1) / (T)(2 * n + 1);
                gr *= inn; gi *= inn; hr *= inn; hi *= inn;
                vr = ((T)n * gr - yr) * t;
                vi = ((T)n * gi - yi) * t;
                wr = ((T)(n + 1) * gr + yr) * t;
                wi = ((T)(n + 1) * gi + yi) * t;
                xr = hr;
                xi = hi;
            }
            if (m == 0) { vi = T(0); wi = T(0); xi = T(0); }
        }
        const int o = n * P1 + m;
        cu[2 * o] = scale * vr; cu[2 * o + 1] = scale * vi;
        cu[2 * (S + o)] = scale * wr; cu[2 * (S + o) + 1] = scale * wi;
        cu[2 * (2 * S + o)] = scale * xr; cu[2 * (2 * S + o) + 1] = scale * xi;
    }
    __syncthreads();
    rotate_vsh(A, cu, cv, v, w, (T)g[0], (T)g[1], (T)g[2], (T)g[3], false);
    T* dst = A.blk + (size_t)e * 6 * S;
    for (int q = tid; q < 6 * S; q += bd) dst[q] = cv[q];
}

// One CTA per target sphere: its entries' blocks summed in list order, then the
// VSH synthesis at its nodes added to out.
template <typename T>
__global__ void fft_synth_kernel(FftArgs<T> A) {
    const int i = blockIdx.x;
    const int e0 = A.near_ptr[i], e1 = A.near_ptr[i + 1];
    if (e1 == e0) return;
    const int p = A.p, P1 = A.P1, nlat = A.nlat, nlon = A.nlon, npn = A.npn, S = P1 * P1;
    const TabLayout& tl = A.tl;
    const T* tab = A.tab;
    const T* ct = tab + tl.o_ct;
    const T* st = tab + tl.o_st;
    const T* cph = tab + tl.o_cph;
    const T* sph = tab + tl.o_sph;
    const T* cmk = tab + tl.o_cmk;
    const T* smk = tab + tl.o_smk;
    const T* Pt = tab + tl.o_P;
    const T* dPt = tab + tl.o_dP;
    const T* mSt = tab + tl.o_mS;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* cf = reinterpret_cast<T*>(smraw);  // [3][P1][P1][2]: Y, G, X
    T* Fh = cf + 6 * S;                   // [3][nlat][P1][2]
    T* f = Fh + 3 * nlat * P1 * 2;        // [3][npn]
    const int tid = threadIdx.x, bd = blockDim.x;
    for (int q = tid; q < S; q += bd) {
        const int n = q / P1;
        T V[2] = {T(0), T(0)}, W[2] = {T(0), T(0)}, X[2] = {T(0), T(0)};
        for (int e = e0; e < e1; ++e) {
            const T* b = A.blk + (size_t)e * 6 * S;
            V[0] += b[2 * q]; V[1] += b[2 * q + 1];
            W[0] += b[2 * (S + q)]; W[1] += b[2 * (S + q) + 1];
            X[0] += b[2 * (2 * S + q)]; X[1] += b[2 * (2 * S + q) + 1];
        }
        // (Y, G, X): phi^Y = -(n+1) V + n W, phi^G = V + W
        cf[2 * q] = -(T)(n + 1) * V[0] + (T)n * W[0];
        cf[2 * q + 1] = -(T)(n + 1) * V[1] + (T)n * W[1];
        cf[2 * (S + q)] = V[0] + W[0];
        cf[2 * (S + q) + 1] = V[1] + W[1];
        cf[2 * (2 * S + q)] = X[0];
        cf[2 * (2 * S + q) + 1] = X[1];
    }
    __syncthreads();
    for (int q = tid; q < 3 * nlat * P1; q += bd) {
        const int c = q / (nlat * P1), r = q - c * nlat * P1, j = r / P1, m = r - j * P1;
        T ar = T(0), ai = T(0);
        for (int n = m; n <= p; ++n) {
            const int o = (m * P1 + n) * nlat + j, oc = 2 * (n * P1 + m);
            const T Yr = cf[oc], Yi = cf[oc + 1];
            const T Gr = cf[2 * S + oc], Gi = cf[2 * S + oc + 1];
            const T Xr = cf[4 * S + oc], Xi = cf[4 * S + oc + 1];
            if (c == 0) {
                ar = fma(Yr, Pt[o], ar);
                ai = fma(Yi, Pt[o], ai);
            } else if (c == 1) {
                ar += Gr * dPt[o] + Xi * mSt[o];
                ai += Gi * dPt[o] - Xr * mSt[o];
            } else {
                ar += -Gi * mSt[o] + Xr * dPt[o];
                ai += Gr * mSt[o] + Xi * dPt[o];
            }
        }
        Fh[2 * q] = ar;
        Fh[2 * q + 1] = ai;
    }
    __syncthreads();
    for (int q = tid; q < 3 * npn; q += bd) {
        const int c = q / npn, r = q - c * npn, j = r / nlon, k = r - j * nlon;
        const T* a = Fh + 2 * ((c * nlat + j) * P1);
        T v = T(0);
        for (int m = 1; m <= p; ++m) {
            v = fma(a[2 * m], cmk[m * nlon + k], v);
            v = fma(-a[2 * m + 1], smk[m * nlon + k], v);
        }
        f[q] = a[0] + T(2) * v;
    }
    __syncthreads();
    for (int q = tid; q < npn; q += bd) {
        const int j = q / nlon, k = q - j * nlon;
        const T c = ct[j], sn = st[j], cp = cph[k], sp = sph[k];
        const T fr = f[q], ft = f[npn + q], fp = f[2 * npn + q];
        double* o = A.out + ((size_t)i * npn + q) * 3;
        o[0] += (double)(fr * sn * cp + ft * c * cp - fp * sp);
        o[1] += (double)(fr * sn * sp + ft * c * sp + fp * cp);
        o[2] += (double)(fr * c - ft * sn);
    }
}

template <typename T>
cudaError_t run_fft(sbie_ctx* c, int kind, const FftArgs<T>& A) {
    const int P1 = A.P1, S = P1 * P1;
    size_t sm = sizeof(T) * 24 * (size_t)S;
    cudaError_t e = cudaFuncSetAttribute(fft_rotate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    fft_rotate_kernel<T><<<A.n_near, 128, sm, c->stream>>>(A); ++c->n_launch;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // channels of the rotated coefficients, one "sphere" per entry (built in
    // FP64; the FP32 copy's rows padded to a multiple of 4)
    if (sizeof(T) == 4)
        e = launch_near_prep_pairs(c, kind, A.n_near, nullptr, reinterpret_cast<const float*>(A.pcoef), c->d_fiota,
                                   c->d_fchan, c->d_fchanf);
    else
        e = launch_near_prep_pairs(c, kind, A.n_near, reinterpret_cast<const double*>(A.pcoef), nullptr, c->d_fiota,
                                   c->d_fchan, nullptr);
    if (e != cudaSuccess) return e;
    sm = fft_eval_smem(c->p, kind, sizeof(T));
    auto eval = kind == 0 ? fft_eval_kernel<T, 0> : (kind == 1 ? fft_eval_kernel<T, 1> : fft_eval_kernel<T, 2>);
    e = cudaFuncSetAttribute(eval, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    eval<<<A.n_near, 128, sm, c->stream>>>(A); ++c->n_launch;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sm = sizeof(T) * (6 * (size_t)S + 3 * c->nlat * P1 * 2 + 3 * (size_t)c->npn);
    e = cudaFuncSetAttribute(fft_synth_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    fft_synth_kernel<T><<<c->n, 256, sm, c->stream>>>(A); ++c->n_launch;
    return cudaGetLastError();
}

}  // namespace

// Discs evaluated together by fft_eval_kernel: enough for one node per thread
// of its 128.
int fft_eval_group(int p) {
    const int nlon = 2 * p + 2;
    return std::min(p + 1, (128 + nlon - 1) / nlon);
}

size_t fft_eval_smem(int p, int kind, size_t elem) {
    const int P1 = p + 1, L = kind == 2 ? p + 2 : p + 1, K = (L + 1) * (L + 1);
    const int nch = kind == 2 ? kTracChannels : kVelChannels;
    const int nlat = p + 1, nlon = 2 * p + 2, npn = nlat * nlon, S = P1 * P1;
    (void)K;
    return elem * ((size_t)fft_eval_group(p) * (L + 1) * nch * 2 + 3 * npn + 3 * nlat * P1 * 2 + 6 * S * 4 + 2 * nlon);
}

cudaError_t launch_near_fft(sbie_ctx* c, Kern op, bool f32, double* out) {
    if (c->n_near == 0) return cudaSuccess;
    const int kind = op == Kern::S ? 0 : (op == Kern::D ? 1 : 2);
    const int nch = kind == 2 ? kTracChannels : kVelChannels;
    auto fill = [&](auto& A) {
        A.p = c->p; A.P1 = c->p + 1; A.L = kind == 2 ? c->p + 2 : c->p + 1; A.K = sh_count(A.L);
        A.npn = c->npn; A.nlat = c->nlat; A.nlon = c->nlon; A.n_near = (int)c->n_near;
        A.G = fft_eval_group(c->p);
        A.tl = c->tl; A.geo = c->d_fgeo;
        A.coef = c->d_coef; A.near_ptr = c->d_near_ptr; A.near_idx = c->d_near_idx;
        A.out = out;
    };
    if (f32) {
        FftArgs<float> A;
        fill(A);
        A.nchs = (nch + 3) / 4 * 4;
        A.tab = c->d_tabf; A.rotp = c->d_rotpf; A.rotm = c->d_rotmf;
        A.pcoef = c->d_fcoeff; A.chan = c->d_fchanf; A.blk = c->d_fblkf;
        return run_fft(c, kind, A);
    }
    FftArgs<double> A;
    fill(A);
    A.nchs = nch;
    A.tab = c->d_tab; A.rotp = c->d_rotp; A.rotm = c->d_rotm;
    A.pcoef = c->d_fcoef; A.chan = c->d_fchan; A.blk = c->d_fblk;
    return run_fft(c, kind, A);
}

}  // namespace sbie
