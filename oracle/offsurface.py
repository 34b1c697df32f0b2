"""Exterior evaluation of the Stokes layer potentials of a VSH expansion on the
unit sphere (Sec. 3.2, Eqs. 3.6-3.11) and of the traction of the single layer
(Sec. 3.3, Eq. 3.18).  Test infrastructure only.

Points are given relative to the source centre and in units of its radius; the
caller scales S by the radius (the kernel is homogeneous of degree -1 and the
area element of degree 2), while D and the traction K are scale free.
"""
import numpy as np

from . import dual, vsh
from .dual import Dual


# ---- radial factors of the r >= 1 branches ---------------------------------

def _S_factors(r):
    """Eqs. 3.6-3.8, r >= 1: S[V] = sV V r^{-n-2};
    S[W] = sW W r^{-n} + n/(4n+2) V (r^{-n-2} - r^{-n}); S[X] = sX X r^{-n-1}."""
    def rp(k):
        return 1.0 / r ** k
    fV = lambda n: n / ((2 * n + 1) * (2 * n + 3)) * rp(n + 2)
    fW = lambda n: (n + 1) / ((2 * n + 1) * (2 * n - 1)) * rp(n)
    fWV = lambda n: n / (4 * n + 2) * (rp(n + 2) - rp(n))
    fX = lambda n: 1.0 / (2 * n + 1) * rp(n + 1)
    return fV, fW, fWV, fX


def _D_factors(r):
    """Eqs. 3.9-3.11, r > 1: D[V] = dV V r^{-n-2};
    D[W] = dW W r^{-n} + 2n(n-1)/(4n+2) V (r^{-n-2} - r^{-n}); D[X] = dX X r^{-n-1}."""
    def rp(k):
        return 1.0 / r ** k
    fV = lambda n: (2 * n * n + 4 * n + 3) / ((2 * n + 1) * (2 * n + 3)) * rp(n + 2)
    fW = lambda n: 2 * (n + 1) * (n - 1) / ((2 * n + 1) * (2 * n - 1)) * rp(n)
    fWV = lambda n: 2 * n * (n - 1) / (4 * n + 2) * (rp(n + 2) - rp(n))
    fX = lambda n: (n - 1) / (2 * n + 1) * rp(n + 1)
    return fV, fW, fWV, fX


def _angles(xh):
    """(cos th, sin th, cos ph, sin ph, r) for a list of 3 coordinates, arrays or Duals."""
    x, y, z = xh
    rho = dual.dsqrt(x * x + y * y)
    r = dual.dsqrt(x * x + y * y + z * z)
    rv = dual.value(rho)
    if np.any(rv == 0.0):
        if isinstance(rho, Dual):
            raise ValueError("dual evaluation on the polar axis")
        safe = np.where(rv > 0, rv, 1.0)
        cp = np.where(rv > 0, dual.value(x) / safe, 1.0)
        sp = np.where(rv > 0, dual.value(y) / safe, 0.0)
    else:
        cp = x / rho
        sp = y / rho
    return z / r, rho / r, cp, sp, r


def _velocity(c, xh, factors):
    ct, st, cp, sp, r = _angles(xh)
    fV, fW, fWV, fX = factors(r)
    return vsh.eval_fields(c, ct, st, cp, sp, fV=fV, fW=fW, fX=fX, fWV=fWV)


def S_velocity(c, xh):
    """Single-layer velocity (unit sphere) of coefficients c at points xh (M, 3), |xh| >= 1."""
    xh = np.asarray(xh, float)
    u = _velocity(c, [xh[:, 0], xh[:, 1], xh[:, 2]], _S_factors)
    return np.stack(u, axis=-1)


def D_velocity(c, xh):
    """Double-layer velocity (unit sphere) of coefficients c at points xh (M, 3), |xh| > 1."""
    xh = np.asarray(xh, float)
    u = _velocity(c, [xh[:, 0], xh[:, 1], xh[:, 2]], _D_factors)
    return np.stack(u, axis=-1)


def S_pressure(c, xh):
    """Pressure of the single layer, r >= 1: only S[W_n^m] carries one,
    p = n Y_n^m r^{-n-1} (Sec. 3.2).  This sign satisfies -Lap u + grad p = 0
    (Eq. 5.1) and matches the Stokeslet pressure (r . f)/(4 pi r^3)."""
    from . import sph
    xh = np.asarray(xh, float)
    ct, st, cp, sp, r = sph.angles_of(xh)
    p = c.shape[1] - 1
    Y, dY, mY = sph.sh_tables(p, ct, st, cp, sp)
    out = np.zeros(len(xh))
    for n in range(1, p + 1):
        for m in range(n + 1):
            eps = 1.0 if m == 0 else 2.0
            out += np.real(eps * n * c[1, n, m] * Y[n][m]) / r ** (n + 1)
    return out


def _rotated_coeffs(c, R):
    """Coefficients, in the frame y' = R y, of the field with coefficients c:
    sigma'(y') = R sigma(R^T y').  Rotation keeps the degree, so analysis of the
    samples on the order-p grid is exact."""
    p = c.shape[1] - 1
    ct, st, cp, sp = vsh.grid_angles(p)
    nodes = np.stack([st * cp, st * sp, ct], axis=-1).reshape(-1, 3)
    vals = vsh.synthesis_at(c, nodes @ R)          # sigma(R^T y')
    return vsh.analysis(vals @ R.T, p)             # R sigma(...)


_RX = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def _traction_direct(c, xh, nrm):
    X = Dual.seed(xh.T)
    u = _velocity(c, X, _S_factors)
    J = np.stack([u[i].d for i in range(3)], axis=0)     # J[i, j] = d u_i / d x_j
    p = S_pressure(c, xh)
    E = J + np.swapaxes(J, 0, 1)
    t = np.einsum("ijm,mj->mi", E, nrm) - p[:, None] * nrm
    return t


def S_traction(c, xh, nrm, pole_tol=1e-3):
    """Traction (grad u + grad u^T - p I) n of the single-layer velocity of c at
    points xh (M, 3), |xh| > 1, with target normals nrm (M, 3) (Eq. 3.18; the
    traction operator K of Eq. 2.22 off the surface).

    grad u is taken by forward-mode dual numbers through the exterior formula
    of Eqs. 3.6-3.8 written in Cartesian coordinates.  Targets within pole_tol
    (in sin theta) of the polar axis are evaluated in a frame rotated by 90
    degrees about x, where the angle derivatives are well conditioned."""
    xh = np.asarray(xh, float)
    nrm = np.asarray(nrm, float)
    st = np.hypot(xh[:, 0], xh[:, 1]) / np.linalg.norm(xh, axis=1)
    near_axis = st < pole_tol
    out = np.zeros_like(xh)
    if np.any(~near_axis):
        out[~near_axis] = _traction_direct(c, xh[~near_axis], nrm[~near_axis])
    if np.any(near_axis):
        cr = _rotated_coeffs(c, _RX)
        tr = _traction_direct(cr, xh[near_axis] @ _RX.T, nrm[near_axis] @ _RX.T)
        out[near_axis] = tr @ _RX
    return out
