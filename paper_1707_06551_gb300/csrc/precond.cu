// Two-body (pair) preconditioner for GMRES on the resistance operator
// 1/2 I + D + N (Eq. 5.19) or the mobility operator 1/2 I + K + L (Eq. 5.8).
//
//   M^{-1} r = H r + Z C^{-1} Z^+ r
//
// Z^+ is the VSH analysis (Sec. 2.1) restricted to degree <= 4 ("low modes",
// 73 real coefficients per sphere) and Z the matching synthesis.  H inverts
// each sphere's own operator above degree 4 (the exterior eigenvalues
// D+ = K- of Theorem 2, the same for both operators) and the
// non-band-limited remainder (1/2 I -> x2), and vanishes on the low modes.
// C^{-1} is an additive Schwarz approximation of the low-mode operator over
// close pairs: for each close pair (i, k) the 146 x 146 system
// [[L_i, B_ik], [B_ki, L_k]] is inverted once, and sphere i averages the
// answers of its pairs (an isolated sphere uses L_i^{-1}).  L_i is the
// sphere's own low-mode block and B_ik the low-mode block of the pair
// coupling (close-pair expansion + completion flow of the operator), either
// probed exactly (the operator applied to each low mode on a two-sphere
// problem) or predicted by the pair network in the pair frame and rotated.
// Each operator has its own blocks (PrecState in the context).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.h"
#include "mlp.h"

namespace sbie {

namespace {

struct Mode {
    int t, n, m, part;
};

std::vector<Mode> low_modes() {
    std::vector<Mode> out;
    for (int t = 0; t < 3; ++t)
        for (int n = 0; n <= kPrecL; ++n) {
            if (t > 0 && n == 0) continue;
            for (int m = 0; m <= n; ++m) {
                out.push_back(Mode{t, n, m, 0});
                if (m >= 1) out.push_back(Mode{t, n, m, 1});
            }
        }
    return out;
}

}  // namespace

// Low-mode synthesis ZS [npn][3][73] and analysis ZA [73][npn][3] on the grid
// of order p, from the Legendre tables (same quadrature as the self kernel).
void lowmode_tables(int p, std::vector<double>& ZS, std::vector<double>& ZA) {
    TabLayout tl = tab_layout(p);
    std::vector<double> tab;
    build_tables(p, tab);
    const std::vector<Mode> modes = low_modes();
    const int NM = (int)modes.size(), npn = tl.npn, P1 = p + 1;
    ZS.assign((size_t)npn * 3 * NM, 0.0);
    ZA.assign((size_t)NM * npn * 3, 0.0);
    for (int j = 0; j < tl.nlat; ++j)
        for (int k = 0; k < tl.nlon; ++k) {
            const int q = j * tl.nlon + k;
            const double ct = tab[tl.o_ct + j], st = tab[tl.o_st + j], cp = tab[tl.o_cph + k], sp = tab[tl.o_sph + k];
            const double w = tab[tl.o_w + j];
            const double er[3] = {st * cp, st * sp, ct}, et[3] = {ct * cp, ct * sp, -st}, ep[3] = {-sp, cp, 0.0};
            for (int b = 0; b < NM; ++b) {
                const Mode& md = modes[b];
                const int n = md.n, m = md.m;
                const int o = (m * P1 + n) * tl.nlat + j;
                const double P = tab[tl.o_P + o], dP = tab[tl.o_dP + o], mS = tab[tl.o_mS + o];
                // spherical components (r, theta, phi) of Z / e^{i m phi}: (real, imag) pairs
                double zr[3][2];
                if (md.t == 0) {  // V = G - (n+1) Y e_r
                    zr[0][0] = -(n + 1.0) * P; zr[0][1] = 0.0;
                    zr[1][0] = dP; zr[1][1] = 0.0;
                    zr[2][0] = 0.0; zr[2][1] = mS;
                } else if (md.t == 1) {  // W = G + n Y e_r
                    zr[0][0] = n * P; zr[0][1] = 0.0;
                    zr[1][0] = dP; zr[1][1] = 0.0;
                    zr[2][0] = 0.0; zr[2][1] = mS;
                } else {  // X = dY e_phi - (i m Y / sin) e_theta
                    zr[0][0] = 0.0; zr[0][1] = 0.0;
                    zr[1][0] = 0.0; zr[1][1] = -mS;
                    zr[2][0] = dP; zr[2][1] = 0.0;
                }
                const double cm = tab[tl.o_cmk + m * tl.nlon + k], sm = tab[tl.o_smk + m * tl.nlon + k];
                double re[3], im[3];  // Cartesian Re Z, Im Z
                for (int c = 0; c < 3; ++c) {
                    double sr = 0, si = 0;
                    for (int a = 0; a < 3; ++a) {
                        const double ea = a == 0 ? er[c] : (a == 1 ? et[c] : ep[c]);
                        // (zr + i zi) (cm + i sm)
                        sr += ea * (zr[a][0] * cm - zr[a][1] * sm);
                        si += ea * (zr[a][0] * sm + zr[a][1] * cm);
                    }
                    re[c] = sr;
                    im[c] = si;
                }
                double norm2 = md.t == 0 ? (n + 1.0) * (2.0 * n + 1.0) : (md.t == 1 ? n * (2.0 * n + 1.0) : n * (n + 1.0));
                for (int c = 0; c < 3; ++c) {
                    double syn, ana;
                    if (md.part == 0) {
                        syn = (m == 0 ? 1.0 : 2.0) * re[c];
                        ana = w * re[c] / norm2;
                    } else {
                        syn = -2.0 * im[c];
                        ana = -w * im[c] / norm2;
                    }
                    ZS[((size_t)q * 3 + c) * NM + b] = syn;
                    ZA[((size_t)b * npn + q) * 3 + c] = ana;
                }
            }
        }
}

// Real low-mode rotation R (73 x 73): coefficients of the field in the frame
// whose axes are the columns of Q, a' = R a.  Block diagonal in (type, n) with
// the scalar rotation of degree n, computed by resampling Y o Q on the grid of
// order 4 (exact: Y o Q has degree n).  The grid, its weights and the
// projections onto the real basis at the grid nodes do not depend on Q and
// are computed once.
namespace {

constexpr int kRL = kPrecL, kRLat = kRL + 1, kRLon = 2 * kRL + 2, kRNodes = kRLat * kRLon;
constexpr int kRSh = (kRL + 1) * (kRL + 1);

// Normalised Pbar_n^m(t) (no Condon-Shortley phase), n <= 4, at one point by
// the normalised three-term recurrence; P[m (L+1) + n].
void pbar_fixed(double t, double s, double* P) {
    for (int i = 0; i < kRSh; ++i) P[i] = 0.0;
    double pmm = 1.0 / std::sqrt(4.0 * kPi);
    for (int m = 0; m <= kRL; ++m) {
        if (m > 0) pmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
        P[m * (kRL + 1) + m] = pmm;
        if (m + 1 <= kRL) P[m * (kRL + 1) + m + 1] = std::sqrt(2.0 * m + 3.0) * t * pmm;
        for (int n = m + 2; n <= kRL; ++n) {
            double a = std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            P[m * (kRL + 1) + n] = a * (t * P[m * (kRL + 1) + n - 1] - b * P[m * (kRL + 1) + n - 2]);
        }
    }
}

struct RotGrid {
    double y[kRNodes][3];
    // w * (projection weight of real coefficient `row` of degree n) at node q:
    // row 0: Y_n0, 2m-1: Re Y_nm, 2m: -Im Y_nm
    double proj[kRL + 1][2 * kRL + 1][kRNodes];
};

const RotGrid& rot_grid() {
    static const RotGrid G = [] {
        RotGrid g{};
        TabLayout tl = tab_layout(kRL);
        std::vector<double> tab;
        build_tables(kRL, tab);
        double P[kRSh];
        for (int j = 0; j < tl.nlat; ++j)
            for (int k = 0; k < tl.nlon; ++k) {
                const int q = j * tl.nlon + k;
                const double ct = tab[tl.o_ct + j], st = tab[tl.o_st + j], cp = tab[tl.o_cph + k], sp = tab[tl.o_sph + k];
                const double w = tab[tl.o_w + j];
                g.y[q][0] = st * cp;
                g.y[q][1] = st * sp;
                g.y[q][2] = ct;
                pbar_fixed(ct, st, P);
                const double phi = std::atan2(sp, cp);
                for (int n = 0; n <= kRL; ++n)
                    for (int m = 0; m <= n; ++m) {
                        const double Py = P[m * (kRL + 1) + n];
                        if (m == 0) {
                            g.proj[n][0][q] = w * Py;
                        } else {
                            g.proj[n][2 * m - 1][q] = w * Py * std::cos(m * phi);
                            g.proj[n][2 * m][q] = -w * Py * std::sin(m * phi);
                        }
                    }
            }
        return g;
    }();
    return G;
}

}  // namespace

namespace {

// D[n][row][mu]: coefficient `row` of the rotated real basis function mu
void lowmode_d(const double Q[9], double (&D)[kRL + 1][2 * kRL + 1][2 * kRL + 1]) {
    const RotGrid& G = rot_grid();
    for (int n = 0; n <= kRL; ++n)
        for (int r = 0; r < 2 * kRL + 1; ++r)
            for (int c = 0; c < 2 * kRL + 1; ++c) D[n][r][c] = 0.0;
    double P[kRSh], vx[2 * kRL + 1];
    for (int q = 0; q < kRNodes; ++q) {
        const double* y = G.y[q];
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = Q[3 * a + 0] * y[0] + Q[3 * a + 1] * y[1] + Q[3 * a + 2] * y[2];
        const double rho = std::sqrt(x[0] * x[0] + x[1] * x[1]);
        const double cpx = rho > 0 ? x[0] / rho : 1.0, spx = rho > 0 ? x[1] / rho : 0.0;
        pbar_fixed(x[2], rho, P);
        // cos / sin (m phi_x) by the angle-addition recurrence
        double cm[kRL + 1], sm[kRL + 1];
        cm[0] = 1.0;
        sm[0] = 0.0;
        for (int m = 1; m <= kRL; ++m) {
            cm[m] = cm[m - 1] * cpx - sm[m - 1] * spx;
            sm[m] = sm[m - 1] * cpx + cm[m - 1] * spx;
        }
        for (int n = 0; n <= kRL; ++n) {
            const int d = 2 * n + 1;
            // values at x of the real basis: Y_n0, 2 Re Y_nm, -2 Im Y_nm
            vx[0] = P[n];
            for (int m = 1; m <= n; ++m) {
                const double Px = P[m * (kRL + 1) + n];
                vx[2 * m - 1] = 2.0 * Px * cm[m];
                vx[2 * m] = -2.0 * Px * sm[m];
            }
            for (int row = 0; row < d; ++row) {
                const double pr = G.proj[n][row][q];
                for (int mu = 0; mu < d; ++mu) D[n][row][mu] += pr * vx[mu];
            }
        }
    }
}

}  // namespace

void lowmode_rotation(const double Q[9], std::vector<double>& R) {
    const int NM = kLowModes;
    double D[kRL + 1][2 * kRL + 1][2 * kRL + 1];
    lowmode_d(Q, D);
    // scatter into R: the same D_n for V, W, X
    R.assign((size_t)NM * NM, 0.0);
    static const std::vector<Mode> modes = low_modes();
    auto sub = [](const Mode& md) { return md.m == 0 ? 0 : (md.part == 0 ? 2 * md.m - 1 : 2 * md.m); };
    for (int a = 0; a < NM; ++a)
        for (int b = 0; b < NM; ++b) {
            const Mode &ma = modes[a], &mb = modes[b];
            if (ma.t != mb.t || ma.n != mb.n) continue;
            R[(size_t)a * NM + b] = D[ma.n][sub(ma)][sub(mb)];
        }
}

void lowmode_rotation_blocks(const double Q[9], float* Dc) {
    double D[kRL + 1][2 * kRL + 1][2 * kRL + 1];
    lowmode_d(Q, D);
    int o = 0;
    for (int n = 0; n <= kPrecL; ++n)
        for (int r = 0; r < 2 * n + 1; ++r)
            for (int c = 0; c < 2 * n + 1; ++c) Dc[o++] = (float)D[n][r][c];
}

namespace {

// ---- device kernels --------------------------------------------------------

// density of problem q: low mode `beta` on local sphere `side` (0 or 1), zero elsewhere
__global__ void probe_density_kernel(int npn, int sph_per_prob, int side, int beta, const double* __restrict__ ZS,
                                     long long N, double* __restrict__ dens) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long sphere = i / npn;
    const int q = (int)(i - sphere * npn);
    const bool on = (int)(sphere % sph_per_prob) == side;
    for (int c = 0; c < 3; ++c) dens[3 * i + c] = on ? ZS[((size_t)q * 3 + c) * kLowModes + beta] : 0.0;
}

// column beta of the low-mode blocks: out[sphere][row][beta] = (ZA . u_sphere)[row]
__global__ void probe_analysis_kernel(int npn, const double* __restrict__ ZA, const double* __restrict__ u, int beta,
                                      double* __restrict__ blocks) {
    const long long sphere = blockIdx.x;
    const int row = threadIdx.x;
    if (row >= kLowModes) return;
    const double* us = u + (size_t)sphere * npn * 3;
    const double* za = ZA + (size_t)row * npn * 3;
    double s = 0.0;
    for (int e = 0; e < npn * 3; ++e) s = fma(za[e], us[e], s);
    blocks[((size_t)sphere * kLowModes + row) * kLowModes + beta] = s;
}

// Probes for G low modes at once: sphere j (its own single-sphere problem)
// carries low mode beta = b0 + j mod G of side 0 (zero when beta >= 73).
__global__ void probe_density_multi_kernel(int npn, int G, int b0, const double* __restrict__ ZS, long long N,
                                           double* __restrict__ dens) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long sphere = i / npn;
    const int q = (int)(i - sphere * npn);
    const int beta = b0 + (int)(sphere % G);
    for (int c = 0; c < 3; ++c) dens[3 * i + c] = beta < kLowModes ? ZS[((size_t)q * 3 + c) * kLowModes + beta] : 0.0;
}

// out[u][row][beta] = (ZA . u_sphere)[row] for sphere j = u G + (beta - b0)
__global__ void probe_analysis_multi_kernel(int npn, int G, int b0, const double* __restrict__ ZA,
                                            const double* __restrict__ u, double* __restrict__ blocks) {
    const long long sphere = blockIdx.x;
    const int row = threadIdx.x;
    const int beta = b0 + (int)(sphere % G);
    if (row >= kLowModes || beta >= kLowModes) return;
    const long long unit = sphere / G;
    const double* us = u + (size_t)sphere * npn * 3;
    const double* za = ZA + (size_t)row * npn * 3;
    double s = 0.0;
    for (int e = 0; e < npn * 3; ++e) s = fma(za[e], us[e], s);
    blocks[((size_t)unit * kLowModes + row) * kLowModes + beta] = s;
}

// Degree, position within its (type, degree) block, and block start of low
// mode a (the modes run type-major, then degree, then m with (Re, Im) pairs).
__device__ __forceinline__ void mode_block(int a, int& n, int& sub, int& start) {
    int t = 0, base = 0;
    const int per[3] = {(kPrecL + 1) * (kPrecL + 1), (kPrecL + 1) * (kPrecL + 1) - 1, (kPrecL + 1) * (kPrecL + 1) - 1};
    while (a - base >= per[t]) base += per[t++];
    int r = a - base;
    n = t == 0 ? 0 : 1;
    while (r >= 2 * n + 1) r -= 2 * n + 1, ++n;
    sub = r;
    start = a - r;
}

// Pair systems [[L_a, B_ab], [B_ba, L_b]] (FP32, 146 x 146) of the learned
// preconditioner, one CTA per pair: the network's pair-frame blocks
// (standardised outputs Y, de-standardised here) turned to the lab frame,
// B = Ri Bp R, with R, Ri block diagonal by (type, degree) and given per
// direction as the compact degree blocks D_n (Dr for R, Di for Ri, 165 values
// each); direction 2q gives B_ba, 2q + 1 gives B_ab.
__global__ void __launch_bounds__(256) pair_system_kernel(const int2* __restrict__ pairs, const int* __restrict__ uid,
                                                          const float* __restrict__ Lu, const float* __restrict__ Y,
                                                          const float* __restrict__ mean, const float* __restrict__ sd,
                                                          const float* __restrict__ Dr, const float* __restrict__ Di,
                                                          float* __restrict__ sys) {
    constexpr int NM = kLowModes, BLK = NM * NM, W = 2 * NM, NDC = 165;
    __shared__ float B[BLK], T[BLK], dr[NDC], di[NDC];
    const int q = blockIdx.x;
    const int2 pr = pairs[q];
    float* M = sys + (size_t)q * W * W;
    const float* La = Lu + (size_t)uid[pr.x] * BLK;
    const float* Lb = Lu + (size_t)uid[pr.y] * BLK;
    for (int e = threadIdx.x; e < BLK; e += blockDim.x) {
        const int r = e / NM, c = e - r * NM;
        M[r * W + c] = La[e];
        M[(NM + r) * W + NM + c] = Lb[e];
    }
    for (int dir = 0; dir < 2; ++dir) {
        const size_t t = 2 * (size_t)q + dir;
        __syncthreads();
        for (int e = threadIdx.x; e < BLK; e += blockDim.x) B[e] = Y[t * BLK + e] * sd[e] + mean[e];
        for (int e = threadIdx.x; e < NDC; e += blockDim.x) {
            dr[e] = Dr[t * NDC + e];
            di[e] = Di[t * NDC + e];
        }
        __syncthreads();
        // T = B R: T[k][s] = sum over l in the block of s of B[k][l] D_n[sub l][sub s]
        for (int e = threadIdx.x; e < BLK; e += blockDim.x) {
            const int k = e / NM, s = e - k * NM;
            int n, ss, st;
            mode_block(s, n, ss, st);
            const int d = 2 * n + 1, off = n * (2 * n - 1) * (2 * n + 1) / 3;
            float v = 0.f;
            for (int j = 0; j < d; ++j) v = fmaf(B[k * NM + st + j], dr[off + j * d + ss], v);
            T[e] = v;
        }
        __syncthreads();
        // out = Ri T: out[r][s] = sum over k in the block of r of Di_n[sub r][sub k] T[k][s]
        for (int e = threadIdx.x; e < BLK; e += blockDim.x) {
            const int r = e / NM, s = e - r * NM;
            int n, sr, st;
            mode_block(r, n, sr, st);
            const int d = 2 * n + 1, off = n * (2 * n - 1) * (2 * n + 1) / 3;
            float v = 0.f;
            for (int j = 0; j < d; ++j) v = fmaf(di[off + sr * d + j], T[(st + j) * NM + s], v);
            if (dir == 0) M[(NM + r) * W + s] = v;   // B_ba
            else M[r * W + NM + s] = v;              // B_ab
        }
    }
}

// own systems: S[i] = L of sphere i's radius
__global__ void own_system_kernel(int n, const int* __restrict__ uid, const float* __restrict__ Lu,
                                  float* __restrict__ S) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int BLK = kLowModes * kLowModes;
    if (e >= (long long)n * BLK) return;
    const long long i = e / BLK;
    S[e] = Lu[(size_t)uid[i] * BLK + (e - i * BLK)];
}

// In-place inverse of `count` n x n matrices (FP32, row-major, contiguous) by
// Gauss-Jordan elimination with partial pivoting in shared memory.  A pivot
// below 1e-30 sets *bad (the matrix is left unchanged in that case).
__global__ void __launch_bounds__(256) gauss_jordan_kernel(int n, float* __restrict__ mats, int* __restrict__ bad) {
    extern __shared__ float sm[];
    const int W = 2 * n;
    float* A = sm;          // [n][2n]
    float* f = sm + n * W;  // [n] elimination multipliers of the current column
    __shared__ int piv;
    __shared__ float pval;
    float* M = mats + (size_t)blockIdx.x * n * n;
    for (int e = threadIdx.x; e < n * W; e += blockDim.x) {
        int r = e / W, c = e - r * W;
        A[e] = c < n ? M[r * n + c] : (c - n == r ? 1.f : 0.f);
    }
    __syncthreads();
    bool ok = true;
    for (int col = 0; col < n; ++col) {
        if (threadIdx.x < 32) {
            float best = -1.f;
            int bi = col;
            for (int r = col + threadIdx.x; r < n; r += 32) {
                float v = fabsf(A[r * W + col]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                float ob = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best) { best = ob; bi = oi; }
            }
            if (threadIdx.x == 0) {
                piv = bi;
                pval = A[bi * W + col];
            }
        }
        __syncthreads();
        if (fabsf(pval) < 1e-30f) {
            ok = false;
            break;
        }
        const int pr = piv;
        if (pr != col)
            for (int c = threadIdx.x; c < W; c += blockDim.x) {
                float t = A[col * W + c];
                A[col * W + c] = A[pr * W + c];
                A[pr * W + c] = t;
            }
        __syncthreads();
        const float inv = 1.f / A[col * W + col];
        __syncthreads();
        for (int c = threadIdx.x; c < W; c += blockDim.x) A[col * W + c] *= inv;
        for (int r = threadIdx.x; r < n; r += blockDim.x) f[r] = (r == col) ? 0.f : A[r * W + col];
        __syncthreads();
        for (int e = threadIdx.x; e < n * W; e += blockDim.x) {
            int r = e / W, c = e - r * W;
            A[e] -= f[r] * A[col * W + c];
        }
        __syncthreads();
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(bad, 1);
        return;
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int r = e / n, c = e - r * n;
        M[e] = A[r * W + n + c];
    }
}

// low-mode real coefficients of every sphere from the VSH coefficients
__global__ void gather_low_kernel(int n_sph, int P1, const double* __restrict__ coef, const int4* __restrict__ modes,
                                  double* __restrict__ low) {
    const int s = blockIdx.x;
    const int b = threadIdx.x;
    if (s >= n_sph || b >= kLowModes) return;
    const int4 md = modes[b];  // t, n, m, part
    const double* cg = coef + (size_t)s * 3 * P1 * P1 * 2;
    const int o = md.y * P1 + md.z;  // coefficient layout [type][n][m] (re, im)
    low[(size_t)s * kLowModes + b] = cg[2 * (md.x * P1 * P1 + o) + md.w];
}

// coarse correction e_i (see the header comment).  One CTA per sphere; each
// warp takes whole matrix rows (rows r = warp, warp + nwarps, ...) and its
// lanes read a row's columns coalesced.  The dot products run in double-float
// arithmetic on the FP32 pipe (GB300 issues FP64 at a small fraction of the
// FP32 rate): a coefficient is split c = ch + cl into floats, m ch is formed
// exactly with an FMA and m cl added rounded, and every sum is a TwoSum, so the
// map stays linear to about 1e-14.  The pair sums of a row are kept as float
// pairs in shared memory (one warp owns each row) and weighted by 1 / deg in
// FP64 once at the end.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_madd(float& h, float& l, float m, float ch, float cl) {
    const float p = m * ch;
    float pe = fmaf(m, ch, -p);
    pe = fmaf(m, cl, pe);
    float sh, se;
    two_sum_f(h, p, sh, se);
    h = sh;
    l += se + pe;
}
// sum of (h, l) over the warp, in every lane
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
    for (int o = 16; o; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        float sh, se;
        two_sum_f(h, oh, sh, se);
        h = sh;
        l = (l + ol) + se;
    }
}
constexpr int kCoarseThreads = 512;
__global__ void coarse_kernel(const int* __restrict__ pp_ptr, const int* __restrict__ pp_idx,
                              const int* __restrict__ pp_pair, const float* __restrict__ pinv,
                              const float* __restrict__ sinv, const double* __restrict__ low, double* __restrict__ e) {
    constexpr int L = kLowModes;
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __shared__ float ch[2 * L], cl[2 * L];   // staged coefficients, split
    __shared__ float ah[L], al[L];           // per-row sums over the pairs
    const int e0 = pp_ptr[i], e1 = pp_ptr[i + 1];
    const int deg = e1 - e0;
    for (int t = threadIdx.x; t < L; t += blockDim.x) ah[t] = al[t] = 0.f;
    // rows of the sphere's own block (no close partner) or of one pair's block
    auto rows = [&](const float* M, int stride, int ncol) {
        for (int r = warp; r < L; r += nw) {
            const float* Mr = M + (size_t)r * stride;
            float h = 0.f, l = 0.f;
            for (int col = lane; col < ncol; col += 32) df_madd(h, l, Mr[col], ch[col], cl[col]);
            df_warp_sum(h, l);
            if (lane == 0) {
                float sh, se;
                two_sum_f(ah[r], h, sh, se);
                ah[r] = sh;
                al[r] += se + l;
            }
        }
    };
    auto stage = [&](int t, double v) {
        const float hi = (float)v;
        ch[t] = hi;
        cl[t] = (float)(v - (double)hi);
    };
    if (deg == 0) {
        for (int t = threadIdx.x; t < L; t += blockDim.x) stage(t, low[(size_t)i * L + t]);
        __syncthreads();
        rows(sinv + (size_t)i * L * L, L, L);
    }
    for (int ee = e0; ee < e1; ++ee) {
        const int k = pp_idx[ee];
        const int a = min(i, k), b = max(i, k);
        __syncthreads();  // the previous pair's coefficients are no longer read
        for (int t = threadIdx.x; t < 2 * L; t += blockDim.x)
            stage(t, t < L ? low[(size_t)a * L + t] : low[(size_t)b * L + t - L]);
        __syncthreads();
        // rows of sphere i in the pair's [2L][2L] block
        rows(pinv + (size_t)pp_pair[ee] * 4 * L * L + (size_t)(i == a ? 0 : L) * 2 * L, 2 * L, 2 * L);
    }
    __syncthreads();
    const double w = deg > 0 ? 1.0 / deg : 1.0;
    for (int t = threadIdx.x; t < L; t += blockDim.x) e[(size_t)i * L + t] = ((double)ah[t] + (double)al[t]) * w;
}

// The coarse correction of the FP32 inner solves: one CTA per directed
// (sphere, pair) entry of the pair lists -- the 73 rows of sphere i in the
// pair's 146 x 146 inverse times the pair's low-mode vector, in FP32 (a fixed
// linear map to FP32 rounding, which the FP32 inner solves tolerate) -- and one
// CTA per sphere without close partners (its own 73 x 73 inverse).  Many more
// CTAs than spheres keep enough loads in flight for the inverses' 48 MB
// (resistance_256) to stream at HBM rate; coarse_average_kernel then averages
// each sphere's entries in a fixed order.
constexpr int kCoarse32Threads = 256;
__global__ void __launch_bounds__(kCoarse32Threads)
    coarse_f32_kernel(int n, int n_entries, const int* __restrict__ pp_ptr, const int* __restrict__ pp_idx,
                      const int* __restrict__ pp_pair, const int* __restrict__ pp_own,
                      const float* __restrict__ pinv, const float* __restrict__ sinv, const double* __restrict__ low,
                      float* __restrict__ part, double* __restrict__ e) {
    constexpr int L = kLowModes;
    __shared__ float cv[2 * L];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* M;
    int stride, ncol, i;
    float* dst = nullptr;
    if (blockIdx.x < n_entries) {
        const int ee = blockIdx.x;
        i = pp_own[ee];
        const int k = pp_idx[ee];
        const int a = min(i, k), b = max(i, k);
        for (int t = threadIdx.x; t < 2 * L; t += blockDim.x)
            cv[t] = (float)(t < L ? low[(size_t)a * L + t] : low[(size_t)b * L + t - L]);
        M = pinv + (size_t)pp_pair[ee] * 4 * L * L + (size_t)(i == a ? 0 : L) * 2 * L;
        stride = ncol = 2 * L;
        dst = part + (size_t)ee * L;
    } else {
        i = blockIdx.x - n_entries;
        if (i >= n || pp_ptr[i + 1] > pp_ptr[i]) return;
        for (int t = threadIdx.x; t < L; t += blockDim.x) cv[t] = (float)low[(size_t)i * L + t];
        M = sinv + (size_t)i * L * L;
        stride = ncol = L;
    }
    __syncthreads();
    for (int r = warp; r < L; r += nw) {
        const float* Mr = M + (size_t)r * stride;
        float acc = 0.f;
#pragma unroll 5
        for (int col = lane; col < ncol; col += 32) acc = fmaf(Mr[col], cv[col], acc);
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            if (dst) dst[r] = acc;
            else e[(size_t)i * L + r] = (double)acc;
        }
    }
}

__global__ void coarse_average_kernel(int n, const int* __restrict__ pp_ptr, const float* __restrict__ part,
                                      double* __restrict__ e) {
    constexpr int L = kLowModes;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * L) return;
    const int i = (int)(t / L), r = (int)(t - (long long)i * L);
    const int e0 = pp_ptr[i], e1 = pp_ptr[i + 1];
    if (e1 == e0) return;  // written by the sphere's own CTA
    float s = 0.f;
    for (int ee = e0; ee < e1; ++ee) s += part[(size_t)ee * L + r];
    e[t] = (double)s / (double)(e1 - e0);
}

// out_sphere += ZS . e_sphere
__global__ void synth_add_kernel(int npn, long long N, const double* __restrict__ ZS, const double* __restrict__ e,
                                 double* __restrict__ out) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long s = i / npn;
    const int q = (int)(i - s * npn);
    const double* es = e + (size_t)s * kLowModes;
    for (int c = 0; c < 3; ++c) {
        const double* z = ZS + ((size_t)q * 3 + c) * kLowModes;
        double v = 0.0;
        for (int b = 0; b < kLowModes; ++b) v = fma(z[b], es[b], v);
        out[3 * i + c] += v;
    }
}

// The same in FP32 for the FP32 inner solves (FP64 would make this small
// contraction FP64-bound on GB300): out_sphere += ZS . e_sphere
__global__ void synth_add_f32_kernel(int npn, long long N, const float* __restrict__ ZS, const double* __restrict__ e,
                                     double* __restrict__ out) {
    __shared__ float es[kLowModes];
    const long long i0 = (long long)blockIdx.x * blockDim.x;
    const long long s0 = i0 / npn;
    long long i = i0 + threadIdx.x;
    const bool valid = i < N;
    if (!valid) i = N - 1;
    const long long s = i / npn;
    const int q = (int)(i - s * npn);
    float v[3] = {0.f, 0.f, 0.f};
    const float* z = ZS + (size_t)q * 3 * kLowModes;
    // the block's spheres one at a time through shared memory
    const long long s1 = min((long long)(i0 + blockDim.x - 1), N - 1) / npn;
    for (long long ss = s0; ss <= s1; ++ss) {
        __syncthreads();
        for (int b = threadIdx.x; b < kLowModes; b += blockDim.x) es[b] = (float)e[(size_t)ss * kLowModes + b];
        __syncthreads();
        if (ss != s) continue;
        for (int b = 0; b < kLowModes; ++b) {
            const float eb = es[b];
            v[0] = fmaf(z[b], eb, v[0]);
            v[1] = fmaf(z[kLowModes + b], eb, v[1]);
            v[2] = fmaf(z[2 * kLowModes + b], eb, v[2]);
        }
    }
    if (!valid) return;
    for (int c = 0; c < 3; ++c) out[3 * i + c] += (double)v[c];
}

}  // namespace

cudaError_t launch_pair_systems(cudaStream_t s, int np, const int2* pairs, const int* uid, const float* Lu,
                                const float* Y, const float* mean, const float* sd, const float* Dr, const float* Di,
                                float* sys) {
    if (np == 0) return cudaSuccess;
    pair_system_kernel<<<np, 256, 0, s>>>(pairs, uid, Lu, Y, mean, sd, Dr, Di, sys);
    return cudaGetLastError();
}

cudaError_t launch_own_systems(cudaStream_t s, int n, const int* uid, const float* Lu, float* S) {
    const long long tot = (long long)n * kLowModes * kLowModes;
    own_system_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, uid, Lu, S);
    return cudaGetLastError();
}

cudaError_t launch_gauss_jordan(cudaStream_t s, int n, int count, float* mats, int* d_bad) {
    if (count == 0) return cudaSuccess;
    size_t sm = sizeof(float) * ((size_t)n * 2 * n + n);
    cudaError_t e = cudaFuncSetAttribute(gauss_jordan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    gauss_jordan_kernel<<<count, 256, sm, s>>>(n, mats, d_bad);
    return cudaGetLastError();
}

cudaError_t launch_probe_density(sbie_ctx* c, int sph_per_prob, int side, int beta, const double* ZS, double* dens) {
    probe_density_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->npn, sph_per_prob, side, beta, ZS,
                                                                                 c->N, dens);
    ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_probe_analysis(sbie_ctx* c, const double* ZA, const double* u, int beta, double* blocks) {
    probe_analysis_kernel<<<c->n, 96, 0, c->stream>>>(c->npn, ZA, u, beta, blocks);
    ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_probe_density_multi(sbie_ctx* c, int G, int b0, const double* ZS, double* dens) {
    probe_density_multi_kernel<<<(unsigned)((c->N + 255) / 256), 256, 0, c->stream>>>(c->npn, G, b0, ZS, c->N, dens);
    ++c->n_launch;
    return cudaGetLastError();
}

cudaError_t launch_probe_analysis_multi(sbie_ctx* c, int G, int b0, const double* ZA, const double* u,
                                        double* blocks) {
    probe_analysis_multi_kernel<<<c->n, 96, 0, c->stream>>>(c->npn, G, b0, ZA, u, blocks);
    ++c->n_launch;
    return cudaGetLastError();
}

std::vector<int4> low_mode_table() {
    std::vector<int4> out;
    for (const Mode& m : low_modes()) out.push_back(make_int4(m.t, m.n, m.m, m.part));
    return out;
}

// M^{-1} v on one part (device vectors of that part): see the header comment.
cudaError_t precond_apply(sbie_ctx* c, int slot, const double* v, double* out, bool f32) {
    const PrecState& P = c->prec[slot];
    const long long n3 = c->N * 3;
    cudaError_t e = cudaSuccess;
    if (f32 && self_gemm_ready(c, kSelfPrec)) {
        // H v (with its 2 v) and the low-mode coefficients in one tensor-core GEMM
        e = launch_self_gemm(c, kSelfPrec, v, out, false);
        if (e != cudaSuccess) return e;
    } else {
        // H v: synthesis of (1/D+ above degree 4, 0 below) minus 2, plus 2 v;
        // the self kernel also leaves the VSH coefficients of v in d_coef
        e = launch_self_precond(c, v, out);
        if (e == cudaSuccess) e = blas_lincomb(c, 2.0, v, 1.0, out, out, n3);
        if (e != cudaSuccess) return e;
        gather_low_kernel<<<c->n, 96, 0, c->stream>>>(c->n, c->p + 1, c->d_coef, c->d_modes, c->d_low);
        ++c->n_launch;
    }
    if (f32 && P.d_pp_own) {
        const int ne = P.n_entries;
        coarse_f32_kernel<<<ne + c->n, kCoarse32Threads, 0, c->stream>>>(c->n, ne, P.d_pp_ptr, P.d_pp_idx,
                                                                         P.d_pp_pair, P.d_pp_own, P.d_pinv, P.d_sinv,
                                                                         c->d_low, P.d_cpart, c->d_lowe);
        ++c->n_launch;
        if (ne > 0) {
            coarse_average_kernel<<<(unsigned)(((long long)c->n * kLowModes + 255) / 256), 256, 0, c->stream>>>(
                c->n, P.d_pp_ptr, P.d_cpart, c->d_lowe);
            ++c->n_launch;
        }
    } else {
        coarse_kernel<<<c->n, kCoarseThreads, 0, c->stream>>>(P.d_pp_ptr, P.d_pp_idx, P.d_pp_pair, P.d_pinv,
                                                              P.d_sinv, c->d_low, c->d_lowe);
        ++c->n_launch;
    }
    if (f32 && c->d_ZSf)
        synth_add_f32_kernel<<<(unsigned)((c->N + 127) / 128), 128, 0, c->stream>>>(c->npn, c->N, c->d_ZSf, c->d_lowe,
                                                                                    out);
    else
        synth_add_kernel<<<(unsigned)((c->N + 127) / 128), 128, 0, c->stream>>>(c->npn, c->N, c->d_ZS, c->d_lowe, out);
    ++c->n_launch;
    return cudaGetLastError();
}

}  // namespace sbie
