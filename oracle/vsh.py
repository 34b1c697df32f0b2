"""Vector spherical harmonic analysis and synthesis on the grid of Eq. 4.2.
Test infrastructure only.

Coefficients of a REAL vector field on the unit sphere are stored for m >= 0
only (the m < 0 ones are their conjugates, Y_n^{-m} = conj(Y_n^m)), as a
complex array c[type, n, m] with type 0 = V, 1 = W, 2 = X and zeros for m > n.
W_0 = X_0 = 0, so c[1, 0, 0] = c[2, 0, 0] = 0.
"""
import numpy as np

from . import quadrature, sph


def grid_angles(p):
    t, lam, theta, phi = quadrature.grid(p)
    ct = np.repeat(t[:, None], 2 * p + 2, axis=1)
    st = np.sqrt(1.0 - ct * ct)
    cp = np.repeat(np.cos(phi)[None, :], p + 1, axis=0)
    sp = np.repeat(np.sin(phi)[None, :], p + 1, axis=0)
    return ct, st, cp, sp


def analysis(F, p):
    """VSH coefficients of order p of the nodal field F (shape ((p+1)(2p+2), 3)
    or (p+1, 2p+2, 3)), defined as a function on the unit sphere.

    Steps (Sec. 2.1, read as an exact projection):
      1. spherical components f_r, f_theta, f_phi at every node;
      2. phi^Y = <f_r, Y>, phi^G = <f_theta e_theta + f_phi e_phi, G>/(n(n+1)),
         phi^X = <F, X>/(n(n+1)), with <f, g> the smooth quadrature of Eq. 4.4
         on the unit sphere applied to f conj(g);
      3. phi^V = (n phi^G - phi^Y)/(2n+1), phi^W = ((n+1) phi^G + phi^Y)/(2n+1)
         (Eqs. 2.13-2.14).
    The grid integrates products of degree <= 2p exactly, so for a field of
    degree <= p this is the exact expansion (2.12)."""
    F = np.asarray(F, float).reshape(p + 1, 2 * p + 2, 3)
    ct, st, cp, sp = grid_angles(p)
    w = quadrature.unit_weights(p)
    Y, dY, mY = sph.sh_tables(p, ct, st, cp, sp)
    er, et, ep = sph.frames(ct, st, cp, sp)
    fr = sum(F[..., i] * er[i] for i in range(3))
    ft = sum(F[..., i] * et[i] for i in range(3))
    fp = sum(F[..., i] * ep[i] for i in range(3))
    c = np.zeros((3, p + 1, p + 1), complex)
    for n in range(p + 1):
        for m in range(n + 1):
            phiY = np.sum(w * fr * np.conj(Y[n][m]))
            if n == 0:
                c[0, 0, 0] = -phiY
                continue
            nn = n * (n + 1.0)
            phiG = np.sum(w * (ft * np.conj(dY[n][m]) + fp * np.conj(mY[n][m]))) / nn
            phiX = np.sum(w * (-ft * np.conj(mY[n][m]) + fp * np.conj(dY[n][m]))) / nn
            c[0, n, m] = (n * phiG - phiY) / (2 * n + 1)
            c[1, n, m] = ((n + 1) * phiG + phiY) / (2 * n + 1)
            c[2, n, m] = phiX
    return c


def eval_fields(c, ct, st, cp, sp, fV=None, fW=None, fX=None, fWV=None):
    """Sum_{n,m} fV(n) c^V V + fW(n) c^W W + fWV(n) c^W V + fX(n) c^X X over all
    m in [-n, n] for a real field (m < 0 terms are conjugates), at points given
    by their angles.  f*(n) default to 1 (fWV to 0).  Returns a Cartesian 3-list."""
    p = c.shape[1] - 1
    one = lambda n: 1.0
    zero = lambda n: 0.0
    fV = fV or one
    fW = fW or one
    fX = fX or one
    fWV = fWV or zero
    Y, V, W, X = sph.vsh_tables(p, ct, st, cp, sp)
    out = [0.0 * ct, 0.0 * ct, 0.0 * ct]
    for n in range(p + 1):
        for m in range(n + 1):
            eps = 1.0 if m == 0 else 2.0
            aV = eps * (fV(n) * c[0, n, m] + fWV(n) * c[1, n, m])
            aW = eps * fW(n) * c[1, n, m] if n > 0 else 0.0
            aX = eps * fX(n) * c[2, n, m] if n > 0 else 0.0
            for i in range(3):
                term = aV * V[n][m][i]
                if n > 0:
                    term = term + aW * W[n][m][i] + aX * X[n][m][i]
                out[i] = out[i] + term
    return [o.real for o in out]


def synthesis(c, p_out=None):
    """Nodal values of the field with coefficients c on the grid of order p_out
    (default: the coefficients' own order), shape ((p+1)(2p+2), 3) (Eq. 2.12)."""
    p = c.shape[1] - 1 if p_out is None else p_out
    ct, st, cp, sp = grid_angles(p)
    F = eval_fields(c, ct, st, cp, sp)
    return np.stack([np.real(f) for f in F], axis=-1).reshape(-1, 3)


def synthesis_at(c, dirs):
    """Field with coefficients c at unit directions dirs (shape (M, 3))."""
    ct, st, cp, sp, r = sph.angles_of(dirs)
    F = eval_fields(c, ct, st, cp, sp)
    return np.stack([np.real(f) for f in F], axis=-1)
