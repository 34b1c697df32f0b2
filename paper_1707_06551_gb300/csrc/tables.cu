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

}  // namespace sbie
