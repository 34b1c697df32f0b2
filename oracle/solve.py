"""Porous-media (Problem 1, Eqs. 5.3-5.4), mobility (Problem 2, Eqs. 5.5-5.8),
squirmer (Problem 4, Eqs. 5.14-5.17) and resistance (Problem 5, Eqs.
5.18-5.19) drivers.  Test infrastructure only.

Readings (the paper defers rho to its reference [9] and does not say how the
rigid motions or forces are read off):
  * rho_k = F_k / (4 pi a^2) + (3 / (8 pi a^4)) T_k x (x - c_k), the rigid-form
    density with int rho = F_k and int (y - c_k) x rho = T_k;
  * mobility: u = sum_k S_k[mu + rho] on Gamma_k (Eq. 5.7), then
    v_k = int u / (4 pi a^2) and w_k = (3 / (8 pi a^4)) int (x - c_k) x u;
  * resistance: right-hand side v_i + w_i x (x - c_i) - u_inf(x) with
    u_inf(x) = u0 + G x; F_k = int psi, T_k = int (y - c_k) x psi.
F and T are the force and torque the particle exerts on the fluid.
"""
import numpy as np

from . import gmres as _gmres
from . import operators as ops


def rho_density(g, F, T):
    F = np.asarray(F, float).reshape(-1, 3)
    T = np.asarray(T, float).reshape(-1, 3)
    out = np.zeros((g.N, 3))
    for k in range(g.n):
        s = g.sl(k)
        a = g.a[k]
        out[s] = F[k] / (4 * np.pi * a * a) + (3.0 / (8 * np.pi * a ** 4)) * np.cross(T[k][None, :], g.x[s] - g.c[k])
    return out


def rigid_projection(g, u):
    """(v_k, w_k) of a nodal field u by the node quadrature."""
    v = np.zeros((g.n, 3))
    w = np.zeros((g.n, 3))
    for k in range(g.n):
        s = g.sl(k)
        a = g.a[k]
        v[k] = np.sum(g.w[s, None] * u[s], axis=0) / (4 * np.pi * a * a)
        w[k] = 3.0 / (8 * np.pi * a ** 4) * np.sum(g.w[s, None] * np.cross(g.x[s] - g.c[k], u[s]), axis=0)
    return v, w


def mobility_rhs(g, F, T):
    rho = rho_density(g, F, T)
    return -(0.5 * rho + ops.layer(g, "K", rho)), rho


def solve_mobility_density(g, rho, tol=1e-10, restart=200, max_iter=1000):
    """Eq. 5.8 for an incident force density rho ([N][3]): solve
    (1/2 I + K + L) mu = -(1/2 I + K) rho, u = S[mu + rho], rigid projection."""
    rho = np.asarray(rho, float).reshape(-1, 3)
    b = -(0.5 * rho + ops.layer(g, "K", rho))
    mu, info = _gmres.gmres(lambda v: ops.apply(g, "mobility", v.reshape(-1, 3)), b.ravel(),
                            tol=tol, restart=restart, max_iter=max_iter)
    mu = mu.reshape(-1, 3)
    u = ops.layer(g, "S", mu + rho)
    v, w = rigid_projection(g, u)
    return v, w, dict(info, mu=mu, u=u)


def solve_mobility(g, F, T, tol=1e-10, restart=200, max_iter=1000):
    return solve_mobility_density(g, rho_density(g, F, T), tol, restart, max_iter)


def resistance_rhs(g, v, w, u0=None, G=None):
    v = np.asarray(v, float).reshape(-1, 3)
    w = np.asarray(w, float).reshape(-1, 3)
    b = np.zeros((g.N, 3))
    for k in range(g.n):
        s = g.sl(k)
        b[s] = v[k][None, :] + np.cross(w[k][None, :], g.x[s] - g.c[k])
    if u0 is not None:
        b -= np.asarray(u0, float)[None, :]
    if G is not None:
        b -= g.x @ np.asarray(G, float).T
    return b


def solve_resistance(g, v, w, u0=None, G=None, tol=1e-10, restart=200, max_iter=1000, rhs=None):
    b = resistance_rhs(g, v, w, u0, G) if rhs is None else np.asarray(rhs, float).reshape(-1, 3)
    psi, info = _gmres.gmres(lambda x: ops.apply(g, "resistance", x.reshape(-1, 3)), b.ravel(),
                             tol=tol, restart=restart, max_iter=max_iter)
    psi = psi.reshape(-1, 3)
    F, T = ops.moments(g, psi)
    return F, T, dict(info, psi=psi)


def solve_porous(g, u0=None, G=None, tol=1e-10, restart=200, max_iter=1000):
    """Problem 1: fixed spheres in the imposed flow u_inf = u0 + G x.
    (1/2 I + S + D) mu = -u_inf (Eq. 5.4); u = u_inf + (S + D) mu (Eq. 5.3).
    F_k = int mu and T_k = int (y - c_k) x mu are the force and torque the
    particle exerts on the fluid (the double layer carries none)."""
    b = resistance_rhs(g, np.zeros((g.n, 3)), np.zeros((g.n, 3)), u0, G)
    mu, info = _gmres.gmres(lambda x: ops.apply(g, "porous", x.reshape(-1, 3)), b.ravel(),
                            tol=tol, restart=restart, max_iter=max_iter)
    mu = mu.reshape(-1, 3)
    F, T = ops.moments(g, mu)
    return F, T, dict(info, mu=mu)


def solve_squirmer(g, slip, tol=1e-10, restart=200, max_iter=1000):
    """Problem 4: force- and torque-free spheres with the prescribed nodal slip
    velocity u_s.  Eq. 5.17 with the conditions of Eq. 5.15 is solved in its
    square form
        (1/2 I + S + D)(mu - P mu) - P mu = u_s,
    P the rigid projection of oracle.operators.rigid_part: the density is
    mu - P mu (so int (mu - P mu) = 0 and int (y - c) x (mu - P mu) = 0, which
    with the double layer carrying no force are Eq. 5.15), and the rigid part
    P mu = v_i + w_i x (x - c_i) gives the velocities: v_i = int mu / (4 pi a^2),
    w_i = (3 / (8 pi a^4)) int (y - c_i) x mu."""
    b = np.asarray(slip, float).reshape(-1, 3)
    mu, info = _gmres.gmres(lambda x: ops.apply(g, "squirmer", x.reshape(-1, 3)), b.ravel(),
                            tol=tol, restart=restart, max_iter=max_iter)
    mu = mu.reshape(-1, 3)
    M0, M1 = ops.moments(g, mu)
    v = M0 / (4 * np.pi * g.a[:, None] ** 2)
    w = 3.0 * M1 / (8 * np.pi * g.a[:, None] ** 4)
    return v, w, dict(info, mu=mu, density=mu - ops.rigid_part(g, mu))


def solve_mhd(g, H0, eta, tol=1e-10, restart=200, max_iter=1000):
    """Problem 3: paramagnetic spheres (eta = (mu - mu0)/(mu + mu0)) in the
    imposed field H0.  The single-layer density q of Eq. 5.13, the Maxwell
    traction f of its exterior field on every sphere, and the rigid motions of
    the mobility problem (Eq. 5.8) with f as the incident force density.
    Returns (F, T, v, w, info): F, T the magnetic force and torque on each
    particle (int f, int (x - c) x f)."""
    from . import laplace
    q, iq = laplace.solve_magnetic(g, H0, eta, tol=tol, restart=restart, max_iter=max_iter)
    f = laplace.maxwell_traction(g, q, H0)
    F, T = ops.moments(g, f)
    v, w, im = solve_mobility_density(g, f, tol, restart, max_iter)
    return F, T, v, w, dict(q=q, traction=f, magnetic=iq, mobility=im)
