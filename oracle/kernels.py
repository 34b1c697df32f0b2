"""Stokes kernels and their smooth-quadrature (Nystrom) sums, viscosity 1.
Test infrastructure only.

  Stokeslet  G_ij(x, y) = (1/8pi) (delta_ij / r + r_i r_j / r^3),      Eq. 2.19
  Stresslet  T_ijk(x, y) = -(3/4pi) r_i r_j r_k / r^5,                  Eq. 2.20
  with r = x - y.
  S[s](x)_i = sum_y G_ij(x, y) s_j(y) w(y)                              Eq. 2.21
  D[m](x)_i = -sum_y T_ijk(x, y) n_k(y) m_j(y) w(y)                     Eq. 2.21 (sign: see below)
  K[s](x)_i = sum_y T_ijk(x, y) n_k(x) s_j(y) w(y)                      Eq. 2.22
with the smooth quadrature of Eq. 4.4 (w the node weights).

Sign of D.  With the stresslet exactly as printed in Eq. 2.20 and r = x - y,
Eq. 2.21 gives a double layer whose jump is D_ext - D_int = -mu (it equals
+mu inside for a constant density).  Theorem 2 (D- = -1 on the constant
field W_1, D+ - D- = 1) and the +1/2 I of the exterior-limit BIEs (Eqs. 5.4,
5.19) need the opposite sign, so D here is the negative of the printed
contraction (equivalently r = y - x in Eq. 2.20).  K is the traction of the
Stokeslet and is used as printed; it matches Eq. 3.18 with the Stokeslet
pressure.
"""
import numpy as np

def _block(n_src):
    """Targets per block so that one (targets x sources x 3) temporary stays near 48 MB."""
    return max(1, min(512, 2_000_000 // max(1, n_src)))


def _pairs(xt, ys):
    r = xt[:, None, :] - ys[None, :, :]
    r2 = np.einsum("tsi,tsi->ts", r, r)
    return r, r2


def stokeslet_sum(xt, ys, dens_w):
    """S of the weighted density dens_w (density times weight) at targets xt."""
    out = np.zeros((len(xt), 3))
    BLOCK = _block(len(ys))
    for b in range(0, len(xt), BLOCK):
        r, r2 = _pairs(xt[b:b + BLOCK], ys)
        rinv = 1.0 / np.sqrt(r2)
        rf = np.einsum("tsi,si->ts", r, dens_w)
        out[b:b + BLOCK] = (np.einsum("ts,si->ti", rinv, dens_w)
                            + np.einsum("ts,tsi->ti", rf * rinv ** 3, r)) / (8.0 * np.pi)
    return out


def stresslet_sum_D(xt, ys, ny, dens_w):
    """D of the weighted density with SOURCE normals ny."""
    out = np.zeros((len(xt), 3))
    BLOCK = _block(len(ys))
    for b in range(0, len(xt), BLOCK):
        r, r2 = _pairs(xt[b:b + BLOCK], ys)
        rf = np.einsum("tsi,si->ts", r, dens_w)
        rn = np.einsum("tsi,si->ts", r, ny)
        out[b:b + BLOCK] = 3.0 / (4.0 * np.pi) * np.einsum("ts,tsi->ti", rf * rn / r2 ** 2.5, r)
    return out


def stresslet_sum_K(xt, nx, ys, dens_w):
    """K of the weighted density with TARGET normals nx (traction of S)."""
    out = np.zeros((len(xt), 3))
    BLOCK = _block(len(ys))
    for b in range(0, len(xt), BLOCK):
        r, r2 = _pairs(xt[b:b + BLOCK], ys)
        rf = np.einsum("tsi,si->ts", r, dens_w)
        rn = np.einsum("tsi,ti->ts", r, nx[b:b + BLOCK])
        out[b:b + BLOCK] = -3.0 / (4.0 * np.pi) * np.einsum("ts,tsi->ti", rf * rn / r2 ** 2.5, r)
    return out


def stokeslet(x, y, f):
    """Velocity at points x (M, 3) of point forces f (3,) at y (3,) (Eq. 2.19)."""
    r = np.asarray(x, float) - np.asarray(y, float)[None, :]
    rn = np.linalg.norm(r, axis=1)
    return (f[None, :] / rn[:, None] + (r @ f)[:, None] * r / rn[:, None] ** 3) / (8.0 * np.pi)


def rotlet(x, y, t):
    """Velocity t x r / (8 pi |r|^3) of a point torque t at y (the completion
    flow of the resistance problem, Problem 5)."""
    r = np.asarray(x, float) - np.asarray(y, float)[None, :]
    rn = np.linalg.norm(r, axis=1)
    return np.cross(t[None, :], r) / (8.0 * np.pi * rn[:, None] ** 3)
