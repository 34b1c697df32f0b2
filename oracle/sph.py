"""Scalar and vector spherical harmonics (Sec. 2.1, Definitions 2.1 and 2.2).
Test infrastructure only.

Every function takes the angles through (cos theta, sin theta, cos phi, sin phi)
so that it works on numpy arrays and on oracle.dual.Dual values alike.

Conventions (read from Eq. 2.1, which uses |m|):
  P_n^m(t) = (1 - t^2)^{m/2} d^m P_n / dt^m   for m >= 0, no Condon-Shortley phase;
  Y_n^m = sqrt((2n+1)/(4 pi)) sqrt((n-m)!/(n+m)!) P_n^m(cos theta) e^{i m phi};
  Y_n^{-m} = conj(Y_n^m).
"""
import math

import numpy as np


def legendre_Q(nmax, t):
    """Q[n][m] = d^m P_n / dt^m (t) for 0 <= m <= n <= nmax (zero for m > n).

    Q_mm = (2m-1)!!, Q_{m+1,m} = (2m+1) t Q_mm and
    (n-m) Q_nm = (2n-1) t Q_{n-1,m} - (n+m-1) Q_{n-2,m}, the Legendre
    recurrence divided by (1 - t^2)^{m/2}."""
    zero = 0.0 * t
    Q = [[zero for _ in range(nmax + 2)] for _ in range(nmax + 2)]
    dfact = 1.0
    for m in range(nmax + 1):
        if m > 0:
            dfact *= 2 * m - 1
        Q[m][m] = zero + dfact
        if m + 1 <= nmax:
            Q[m + 1][m] = (2 * m + 1) * dfact * t
        for n in range(m + 2, nmax + 1):
            Q[n][m] = ((2 * n - 1) * t * Q[n - 1][m] - (n + m - 1) * Q[n - 2][m]) * (1.0 / (n - m))
    return Q


def norm_nm(n, m):
    """sqrt((2n+1)/(4 pi)) sqrt((n-|m|)!/(n+|m|)!) of Eq. 2.1."""
    m = abs(m)
    return math.sqrt((2 * n + 1) / (4.0 * math.pi) * math.factorial(n - m) / math.factorial(n + m))


def sh_tables(nmax, ct, st, cp, sp):
    """For 0 <= m <= n <= nmax return lists Y[n][m], dY[n][m], mY[n][m]:
    Y_n^m, d(Y_n^m)/d(theta) and i m Y_n^m / sin(theta) (Eq. 2.1 and the
    surface gradient of Definition 2.2).

    With P_n^m = sin^m Q_nm:
      dP_n^m/dtheta = m cos sin^{m-1} Q_nm - sin^{m+1} Q_{n,m+1},
      P_n^m / sin  = sin^{m-1} Q_nm  (m >= 1),
    so nothing is divided by sin(theta)."""
    Q = legendre_Q(nmax + 1, ct)
    spow = [0.0 * st + 1.0]
    for m in range(1, nmax + 2):
        spow.append(spow[-1] * st)
    e1 = cp + 1j * sp
    E = [0.0 * e1 + 1.0]
    for m in range(1, nmax + 1):
        E.append(E[-1] * e1)
    Y = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    dY = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    mY = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    for n in range(nmax + 1):
        for m in range(n + 1):
            c = norm_nm(n, m)
            Y[n][m] = c * spow[m] * Q[n][m] * E[m]
            if m == 0:
                dY[n][m] = -c * spow[1] * Q[n][1] * E[0]
                mY[n][m] = 0.0 * Y[n][m]
            else:
                dY[n][m] = c * (m * ct * spow[m - 1] * Q[n][m] - spow[m + 1] * Q[n][m + 1]) * E[m]
                mY[n][m] = (1j * m * c) * spow[m - 1] * Q[n][m] * E[m]
    return Y, dY, mY


def frames(ct, st, cp, sp):
    """Cartesian components of e_r, e_theta, e_phi (lists of 3)."""
    zero = 0.0 * ct
    er = [st * cp, st * sp, ct]
    et = [ct * cp, ct * sp, -1.0 * st]
    ep = [-1.0 * sp, cp, zero]
    return er, et, ep


def vsh_tables(nmax, ct, st, cp, sp):
    """Vector spherical harmonics of Definition 2.2 (Eqs. 2.4-2.6) as Cartesian
    3-lists, for 0 <= m <= n <= nmax:
      G = grad_gamma Y = dY/dtheta e_theta + (i m Y / sin theta) e_phi,
      V = G - (n+1) Y e_r,  W = G + n Y e_r,
      X = e_r x G = dY/dtheta e_phi - (i m Y / sin theta) e_theta.
    Returns (Y, V, W, X) as nested lists [n][m]."""
    Y, dY, mY = sh_tables(nmax, ct, st, cp, sp)
    er, et, ep = frames(ct, st, cp, sp)
    V = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    W = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    X = [[None] * (nmax + 1) for _ in range(nmax + 1)]
    for n in range(nmax + 1):
        for m in range(n + 1):
            G = [dY[n][m] * et[i] + mY[n][m] * ep[i] for i in range(3)]
            V[n][m] = [G[i] - (n + 1) * Y[n][m] * er[i] for i in range(3)]
            W[n][m] = [G[i] + n * Y[n][m] * er[i] for i in range(3)]
            X[n][m] = [dY[n][m] * ep[i] - mY[n][m] * et[i] for i in range(3)]
    return Y, V, W, X


def angles_of(xyz):
    """(cos theta, sin theta, cos phi, sin phi, r) of points xyz (shape (..., 3)),
    angles about the origin; phi := 0 on the polar axis."""
    xyz = np.asarray(xyz, float)
    r = np.linalg.norm(xyz, axis=-1)
    rho = np.hypot(xyz[..., 0], xyz[..., 1])
    ct = xyz[..., 2] / r
    st = rho / r
    safe = rho > 0
    cp = np.where(safe, xyz[..., 0] / np.where(safe, rho, 1.0), 1.0)
    sp = np.where(safe, xyz[..., 1] / np.where(safe, rho, 1.0), 0.0)
    return ct, st, cp, sp, r
