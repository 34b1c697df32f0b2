"""Laplace layer potentials on N spheres and the magnetostatic problem of the
multiphysics case study.  Test infrastructure only.

  G^L(x, y) = 1 / (4 pi |x - y|)                                         Eq. 2.18
  S^L[q](x) = int G^L q,   D^L[m](x) = int dG^L/dn(y) m,
  K^L[q](x) = n(x) . grad_x S^L[q](x)  (the flux of Sec. 3.3, Eq. 3.16).
With r = x - y:  dG^L/dn(y) = n(y) . r / (4 pi |r|^3),  grad_x G^L = -r / (4 pi |r|^3).

Self terms by Theorem 1 (Eq. 3.5) on the unit sphere: S^L 1/(2n+1) (times the
radius a: the kernel has degree -1, the area element degree 2), D^L and K^L as
principal values (limits averaged): D+^L = n/(2n+1), D-^L = -(n+1)/(2n+1), and
K^L, the adjoint of D^L on the sphere, has K+^L = D-^L and K-^L = D+^L (the
limits of d/dr of Eq. 3.3), so both principal values are -1/(2(2n+1)).
The exterior limit of grad S^L[Y_n^m] on the unit sphere is
  -(n+1)/(2n+1) Y e_r + 1/(2n+1) grad_gamma Y = V_n^m / (2n+1)
(Eq. 3.3 differentiated; V of Definition 2.2), scale free.
Close pairs use the exterior expansions of Eqs. 3.3-3.4 at r = |x - c|/a; the
flux and the gradient are taken by forward-mode dual numbers.

Problem 3 (Eqs. 5.9-5.13): phi = -H0 . x + S^L[q] with
  (1/2 I + eta K^L) q = eta H0 . n,   eta = (mu - mu0) / (mu + mu0),
K^L the principal value on every sphere's surface.  Readings: the field outside
is H = -grad phi = H0 - grad S^L[q] (exterior limit), and the magnetic traction
on a particle is the Maxwell stress of that field (permeability mu0 = 1),
  f = (H . n) H - |H|^2 n / 2,
which becomes the incident force density rho of the mobility problem (Eq. 5.8).
"""
import numpy as np

from . import dual, gmres as _gmres, quadrature, sph, vsh
from .dual import Dual


def _block(n_src):
    return max(1, min(512, 2_000_000 // max(1, n_src)))


# ---- smooth-quadrature sums (Eq. 4.4) --------------------------------------

def sum_S(xt, ys, qw):
    """S^L of the weighted scalar density qw (density times node weight)."""
    out = np.zeros(len(xt))
    B = _block(len(ys))
    for b in range(0, len(xt), B):
        r = xt[b:b + B, None, :] - ys[None, :, :]
        out[b:b + B] = (qw[None, :] / np.sqrt(np.einsum("tsi,tsi->ts", r, r))).sum(axis=1) / (4 * np.pi)
    return out


def sum_D(xt, ys, ny, qw):
    """D^L with source normals ny."""
    out = np.zeros(len(xt))
    B = _block(len(ys))
    for b in range(0, len(xt), B):
        r = xt[b:b + B, None, :] - ys[None, :, :]
        r2 = np.einsum("tsi,tsi->ts", r, r)
        rn = np.einsum("tsi,si->ts", r, ny)
        out[b:b + B] = (qw[None, :] * rn / r2 ** 1.5).sum(axis=1) / (4 * np.pi)
    return out


def sum_grad(xt, ys, qw):
    """grad_x S^L: shape (targets, 3)."""
    out = np.zeros((len(xt), 3))
    B = _block(len(ys))
    for b in range(0, len(xt), B):
        r = xt[b:b + B, None, :] - ys[None, :, :]
        r2 = np.einsum("tsi,tsi->ts", r, r)
        out[b:b + B] = -np.einsum("ts,tsi->ti", qw[None, :] / r2 ** 1.5, r) / (4 * np.pi)
    return out


# ---- scalar harmonic analysis and synthesis on the grid of Eq. 4.2 ----------

def analysis(f, p):
    """Coefficients c[n, m] (m >= 0, complex) of the real nodal function f on
    the unit sphere: c = sum w f conj(Y_n^m), exact for degree <= p."""
    f = np.asarray(f, float).reshape(p + 1, 2 * p + 2)
    ct, st, cp, sp = vsh.grid_angles(p)
    w = quadrature.unit_weights(p)
    Y, _, _ = sph.sh_tables(p, ct, st, cp, sp)
    c = np.zeros((p + 1, p + 1), complex)
    for n in range(p + 1):
        for m in range(n + 1):
            c[n, m] = np.sum(w * f * np.conj(Y[n][m]))
    return c


def synthesis(c, ct, st, cp, sp, fac=None):
    """sum_n fac(n) sum_m c Y (real field: m < 0 terms conjugate)."""
    p = c.shape[0] - 1
    fac = fac or (lambda n: 1.0)
    Y, _, _ = sph.sh_tables(p, ct, st, cp, sp)
    out = 0.0 * ct
    for n in range(p + 1):
        for m in range(n + 1):
            eps = 1.0 if m == 0 else 2.0
            out = out + eps * fac(n) * c[n, m] * Y[n][m]
    return out.real


def signature(op, n):
    """Theorem 1 on the unit sphere (D and K as principal values)."""
    if op == "SL":
        return 1.0 / (2 * n + 1)
    if op in ("DL", "KL"):
        return -1.0 / (2 * (2 * n + 1))
    raise ValueError(op)


# ---- exterior expansions (Eqs. 3.3-3.4), r >= 1 in source units ------------

def _ext(c, X, fac):
    x, y, z = X
    if not isinstance(x, Dual):  # values: angles_of handles the polar axis
        ct, st, cp, sp, r = sph.angles_of(np.stack([x, y, z], axis=-1))
        return synthesis(c, ct, st, cp, sp, fac=lambda n: fac(n) / r ** (n + 1))
    rho = dual.dsqrt(x * x + y * y)
    r = dual.dsqrt(x * x + y * y + z * z)
    return synthesis(c, z / r, rho / r, x / rho, y / rho, fac=lambda n: fac(n) / r ** (n + 1))


def ext_S(c, xh):
    xh = np.asarray(xh, float)
    return _ext(c, [xh[:, 0], xh[:, 1], xh[:, 2]], lambda n: 1.0 / (2 * n + 1))


def ext_D(c, xh):
    xh = np.asarray(xh, float)
    return _ext(c, [xh[:, 0], xh[:, 1], xh[:, 2]], lambda n: n / (2.0 * n + 1))


def _ext_grad(c, xh):
    X = Dual.seed(xh.T)
    u = _ext(c, X, lambda n: 1.0 / (2 * n + 1))
    return np.asarray(u.d).T


_RX = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def _rotated(c, R):
    """Coefficients, in the frame y' = R y, of the function with coefficients c
    (resampled on the grid: rotation keeps the degree, so this is exact)."""
    p = c.shape[0] - 1
    ct, st, cp, sp = vsh.grid_angles(p)
    nodes = np.stack([st * cp, st * sp, ct], axis=-1).reshape(-1, 3)
    ct2, st2, cp2, sp2, _ = sph.angles_of(nodes @ R)   # R^T y'
    return analysis(synthesis(c, ct2, st2, cp2, sp2), p)


def ext_grad_S(c, xh, pole_tol=1e-3):
    """grad of the exterior S^L expansion at xh (source units), by dual numbers
    through the Cartesian form; targets within pole_tol (in sin theta) of the
    source's polar axis are evaluated in a frame rotated by 90 degrees about x."""
    xh = np.asarray(xh, float)
    st = np.hypot(xh[:, 0], xh[:, 1]) / np.linalg.norm(xh, axis=1)
    near_axis = st < pole_tol
    out = np.zeros_like(xh)
    if np.any(~near_axis):
        out[~near_axis] = _ext_grad(c, xh[~near_axis])
    if np.any(near_axis):
        out[near_axis] = _ext_grad(_rotated(c, _RX), xh[near_axis] @ _RX.T) @ _RX
    return out


# ---- operators ---------------------------------------------------------------

def coefficients(g, q):
    return [analysis(q[g.sl(i)], g.p) for i in range(g.n)]


def layer(g, op, q, targets=None):
    """sum_k S_k^L, D_k^L or K_k^L of the scalar nodal density q at every node
    (self by Theorem 1, far by Eq. 4.4, close pairs by the exterior expansions)."""
    q = np.asarray(q, float).reshape(-1)
    tg = range(g.n) if targets is None else list(targets)
    coefs = coefficients(g, q)
    out = np.zeros(g.N)
    qw = q * g.w
    ct, st, cp, sp = vsh.grid_angles(g.p)
    for i in tg:
        s = g.sl(i)
        # self
        fac = (lambda n: g.a[i] * signature("SL", n)) if op == "SL" else (lambda n: signature(op, n))
        out[s] = synthesis(coefs[i], ct, st, cp, sp, fac=fac).reshape(-1)
        # far
        excl = set(g.near[i]) | {i}
        src = [k for k in range(g.n) if k not in excl]
        if src:
            idx = np.concatenate([np.arange(g.sl(k).start, g.sl(k).stop) for k in src])
            xt = g.x[s]
            if op == "SL":
                out[s] += sum_S(xt, g.x[idx], qw[idx])
            elif op == "DL":
                out[s] += sum_D(xt, g.x[idx], g.nrm[idx], qw[idx])
            else:
                out[s] += np.sum(g.nrm[s] * sum_grad(xt, g.x[idx], qw[idx]), axis=1)
        # close pairs
        for k in g.near[i]:
            xh = (g.x[s] - g.c[k][None, :]) / g.a[k]
            if op == "SL":
                out[s] += g.a[k] * ext_S(coefs[k], xh)
            elif op == "DL":
                out[s] += ext_D(coefs[k], xh)
            else:
                out[s] += np.sum(g.nrm[s] * ext_grad_S(coefs[k], xh), axis=1)
    return out


def grad_S_exterior(g, q):
    """Exterior limit of grad S^L[q] at every node ([N][3]): the own sphere's
    V-mode field sum c/(2n+1) V_n^m, the far field by Eq. 4.4, close pairs by
    the differentiated exterior expansion."""
    q = np.asarray(q, float).reshape(-1)
    coefs = coefficients(g, q)
    out = np.zeros((g.N, 3))
    qw = q * g.w
    for i in range(g.n):
        s = g.sl(i)
        cv = np.zeros((3, g.p + 1, g.p + 1), complex)
        for n in range(g.p + 1):
            cv[0, n, :] = coefs[i][n, :] / (2 * n + 1)
        out[s] = vsh.synthesis(cv)
        excl = set(g.near[i]) | {i}
        src = [k for k in range(g.n) if k not in excl]
        if src:
            idx = np.concatenate([np.arange(g.sl(k).start, g.sl(k).stop) for k in src])
            out[s] += sum_grad(g.x[s], g.x[idx], qw[idx])
        for k in g.near[i]:
            out[s] += ext_grad_S(coefs[k], (g.x[s] - g.c[k][None, :]) / g.a[k])
    return out


def magnetic_operator(g, q, eta):
    """(1/2 I + eta K^L) q (Eq. 5.13)."""
    return 0.5 * np.asarray(q, float).reshape(-1) + eta * layer(g, "KL", q)


def solve_magnetic(g, H0, eta, tol=1e-12, restart=200, max_iter=1000):
    """Single-layer density q of Eq. 5.13 for the imposed field H0."""
    H0 = np.asarray(H0, float)
    b = eta * (g.nrm @ H0)
    q, info = _gmres.gmres(lambda v: magnetic_operator(g, v, eta), b, tol=tol, restart=restart, max_iter=max_iter)
    return q, info


def maxwell_traction(g, q, H0):
    """f = (H . n) H - |H|^2 n / 2 with H = H0 - grad S^L[q] outside ([N][3])."""
    H = np.asarray(H0, float)[None, :] - grad_S_exterior(g, q)
    Hn = np.sum(H * g.nrm, axis=1)
    return Hn[:, None] * H - 0.5 * np.sum(H * H, axis=1)[:, None] * g.nrm
