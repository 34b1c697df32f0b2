// Host-side FP64 tables for one VSH order p: the grid of Eq. 4.2, the smooth
// weights of Eq. 4.4 and normalised associated Legendre functions (Eq. 2.1).
#include <cmath>

#include "common.h"

namespace sbie {


// Gauss-Legendre nodes (descending) and weights by Newton's method on P_n,
// started from the Tricomi-type guess cos(pi (i + 3/4) / (n + 1/2)).
static void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& w) {
    t.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p0 = 1.0; p1 = x; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        t[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

// Normalised Pbar_n^m = sqrt((2n+1)/(4pi) (n-m)!/(n+m)!) P_n^m (no Condon-
// Shortley phase) and Sbar_n^m = Pbar_n^m / sin(theta) (m >= 1) by the
// normalised three-term recurrences
//   Pbar_m^m = sqrt((2m+1)/(2m)) sin Pbar_{m-1}^{m-1},  Pbar_{m+1}^m = sqrt(2m+3) t Pbar_m^m,
//   Pbar_n^m = a_nm (t Pbar_{n-1}^m - b_nm Pbar_{n-2}^m),
//   a_nm = sqrt((4n^2-1)/(n^2-m^2)), b_nm = sqrt(((n-1)^2-m^2)/(4(n-1)^2-1));
// Sbar obeys the same recurrence in n with Sbar_m^m = sqrt((2m+1)/(2m)) Pbar_{m-1}^{m-1}.
// d/dtheta Pbar_n^m = (sqrt((n+m)(n-m+1)) Pbar_n^{m-1} - sqrt((n-m)(n+m+1)) Pbar_n^{m+1}) / 2
// for m >= 1 and -sqrt(n(n+1)) Pbar_n^1 for m = 0.
static void legendre_col(int p, double t, double s, std::vector<double>& P, std::vector<double>& S) {
    // P, S indexed [m][n] with size (p+2) x (p+2)
    int L = p + 1;
    P.assign((L + 1) * (L + 1), 0.0);
    S.assign((L + 1) * (L + 1), 0.0);
    auto at = [L](int m, int n) { return m * (L + 1) + n; };
    double pmm = 1.0 / std::sqrt(4.0 * kPi);
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            double prev = pmm;
            pmm = std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * prev;
            S[at(m, m)] = std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * prev;
        }
        P[at(m, m)] = pmm;
        if (m + 1 <= L) {
            P[at(m, m + 1)] = std::sqrt(2.0 * m + 3.0) * t * pmm;
            S[at(m, m + 1)] = std::sqrt(2.0 * m + 3.0) * t * S[at(m, m)];
        }
        for (int n = m + 2; n <= L; ++n) {
            double a = std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            P[at(m, n)] = a * (t * P[at(m, n - 1)] - b * P[at(m, n - 2)]);
            S[at(m, n)] = a * (t * S[at(m, n - 1)] - b * S[at(m, n - 2)]);
        }
    }
}

void build_tables(int p, std::vector<double>& h) {
    TabLayout tl = tab_layout(p);
    h.assign(tl.total, 0.0);
    std::vector<double> t, lam;
    gauss_legendre(p + 1, t, lam);
    for (int j = 0; j < tl.nlat; ++j) {
        h[tl.o_ct + j] = t[j];
        h[tl.o_st + j] = std::sqrt(1.0 - t[j] * t[j]);
        h[tl.o_w + j] = 2.0 * kPi * lam[j] / (2.0 * p + 2.0);
    }
    for (int k = 0; k < tl.nlon; ++k) {
        double ph = 2.0 * kPi * k / tl.nlon;
        h[tl.o_cph + k] = std::cos(ph);
        h[tl.o_sph + k] = std::sin(ph);
        for (int m = 0; m <= p; ++m) {
            // reduce m k mod nlon for exact periodicity
            double a = 2.0 * kPi * ((m * k) % tl.nlon) / tl.nlon;
            h[tl.o_cmk + m * tl.nlon + k] = std::cos(a);
            h[tl.o_smk + m * tl.nlon + k] = std::sin(a);
        }
    }
    std::vector<double> P, S;
    int L = p + 1;
    auto at = [L](int m, int n) { return m * (L + 1) + n; };
    for (int j = 0; j < tl.nlat; ++j) {
        double tj = h[tl.o_ct + j], sj = h[tl.o_st + j];
        legendre_col(p, tj, sj, P, S);
        for (int m = 0; m <= p; ++m) {
            for (int n = m; n <= p; ++n) {
                int o = (m * (p + 1) + n) * tl.nlat + j;
                h[tl.o_P + o] = P[at(m, n)];
                double d;
                if (m == 0) {
                    d = -std::sqrt((double)n * (n + 1.0)) * (n >= 1 ? P[at(1, n)] : 0.0);
                } else {
                    double up = (m + 1 <= n) ? P[at(m + 1, n)] : 0.0;
                    d = 0.5 * (std::sqrt((double)(n + m) * (n - m + 1.0)) * P[at(m - 1, n)] -
                               std::sqrt((double)(n - m) * (n + m + 1.0)) * up);
                }
                h[tl.o_dP + o] = d;
                h[tl.o_mS + o] = (m == 0) ? 0.0 : m * S[at(m, n)];
            }
        }
    }
}

// Matrices of f -> f o R_x(+90 deg) and f -> f o R_x(-90 deg) on the spherical
// harmonics of each degree n <= p (normalised, no Condon-Shortley phase,
// Y_n^{-m} = conj(Y_n^m)): Y_n^m(R y) = sum_{m'} M_{m' m} Y_n^{m'}(y), m, m' in
// [-n, n], with R_x(+90) (x, y, z) = (x, -z, y).  Computed by projection with the
// quadrature of the order-p grid (exact for degree 2n <= 2p).  Layout: degree
// blocks of (2n+1)^2 complex entries (re, im), row m' + n, column m + n, block n
// starting at n (2n-1)(2n+1)/3.
void rotx90_tables(int p, std::vector<double>& Mp, std::vector<double>& Mm) {
    const TabLayout tl = tab_layout(p);
    std::vector<double> h;
    build_tables(p, h);
    const int nlat = tl.nlat, nlon = tl.nlon, npn = tl.npn, L = p + 1;
    auto at = [L](int m, int n) { return m * (L + 1) + n; };
    size_t total = 0;
    for (int n = 0; n <= p; ++n) total += (size_t)(2 * n + 1) * (2 * n + 1);
    Mp.assign(2 * total, 0.0);
    Mm.assign(2 * total, 0.0);
    // Y_n^m (m >= 0) at the grid nodes and at the rotated nodes
    struct C { double re, im; };
    std::vector<C> Yg((size_t)npn * (p + 1) * (p + 1)), Yp(Yg.size()), Ym(Yg.size());
    auto idx = [p](int q, int n, int m) { return ((size_t)q * (p + 1) + n) * (p + 1) + m; };
    std::vector<double> P, S;
    auto fill = [&](std::vector<C>& Y, int q, double x, double y, double z) {
        const double s = std::sqrt(x * x + y * y);
        const double ph = (s > 0.0) ? std::atan2(y, x) : 0.0;
        legendre_col(p, z, s, P, S);
        for (int n = 0; n <= p; ++n)
            for (int m = 0; m <= n; ++m) {
                const double pv = P[at(m, n)];
                Y[idx(q, n, m)] = {pv * std::cos(m * ph), pv * std::sin(m * ph)};
            }
    };
    for (int j = 0; j < nlat; ++j)
        for (int k = 0; k < nlon; ++k) {
            const int q = j * nlon + k;
            const double st = h[tl.o_st + j], ct = h[tl.o_ct + j], cp = h[tl.o_cph + k], sp = h[tl.o_sph + k];
            const double x = st * cp, y = st * sp, z = ct;
            fill(Yg, q, x, y, z);
            fill(Yp, q, x, -z, y);   // R_x(+90) y
            fill(Ym, q, x, z, -y);   // R_x(-90) y
        }
    // Y_n^m for any sign of m from the stored m >= 0 values
    auto Yv = [&](const std::vector<C>& Y, int q, int n, int m) -> C {
        const C v = Y[idx(q, n, m < 0 ? -m : m)];
        return m < 0 ? C{v.re, -v.im} : v;
    };
    size_t off = 0;
    for (int n = 0; n <= p; ++n) {
        const int w = 2 * n + 1;
        for (int mr = -n; mr <= n; ++mr)
            for (int mc = -n; mc <= n; ++mc) {
                double pr = 0, pi = 0, mr_ = 0, mi = 0;
                for (int j = 0; j < nlat; ++j) {
                    const double wj = h[tl.o_w + j];
                    for (int k = 0; k < nlon; ++k) {
                        const int q = j * nlon + k;
                        const C g = Yv(Yg, q, n, mr);  // conj taken below
                        const C a = Yv(Yp, q, n, mc), b = Yv(Ym, q, n, mc);
                        // a conj(g), b conj(g)
                        pr += wj * (a.re * g.re + a.im * g.im);
                        pi += wj * (a.im * g.re - a.re * g.im);
                        mr_ += wj * (b.re * g.re + b.im * g.im);
                        mi += wj * (b.im * g.re - b.re * g.im);
                    }
                }
                const size_t e = off + (size_t)(mr + n) * w + (mc + n);
                Mp[2 * e] = pr;
                Mp[2 * e + 1] = pi;
                Mm[2 * e] = mr_;
                Mm[2 * e + 1] = mi;
            }
        off += (size_t)w * w;
    }
}

}  // namespace sbie
