"""Pins of the oracle's Laplace family (Sec. 2.2, 3.1, 3.3) and of the
magnetostatic problem (Problem 3, Eqs. 5.9-5.13) against what fixes them
independently: Theorem 1 by high-order quadrature at the pole, the exterior
expansions against upsampled smooth quadrature, a permeable sphere in a
uniform field (closed form), zero net magnetic force on one sphere, the
dipole-dipole forces of two spheres far apart, and the exact discrete
equivalence of the mobility problem for incident densities with equal
moments."""
import math

import numpy as np
import pytest

from oracle import laplace, operators as ops, quadrature, solve as osolve, sph

NT, NP = 96, 64


@pytest.mark.parametrize("n,m", [(n, m) for n in range(5) for m in (0, 1) if m <= n])
def test_theorem_1_by_pole_quadrature(n, m):
    """Target at the north pole of the unit sphere: S^L[Y] = Y/(2n+1); the
    principal values of D^L (source normal) and K^L (target normal) are both
    -Y/(2(2n+1)).  Kernel x area element is bounded there (r = 2 sin(t/2))."""
    u, wu = np.polynomial.legendre.leggauss(NT)
    th = 0.5 * np.pi * (u + 1.0)
    wth = 0.5 * np.pi * wu
    ph = 2 * np.pi * np.arange(NP) / NP
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    ct, st, cp, sp = np.cos(TH), np.sin(TH), np.cos(PH), np.sin(PH)
    Y, _, _ = sph.sh_tables(n, ct, st, cp, sp)
    y = np.stack([st * cp, st * sp, ct], -1)
    dA = (wth[:, None] * st) * (2 * np.pi / NP)
    r = np.array([0.0, 0.0, 1.0]) - y
    rn = np.linalg.norm(r, axis=-1)
    S = np.sum(dA * Y[n][m] / (4 * np.pi * rn))
    D = np.sum(dA * Y[n][m] * np.einsum("abi,abi->ab", r, y) / (4 * np.pi * rn ** 3))
    K = np.sum(dA * Y[n][m] * (-r[..., 2]) / (4 * np.pi * rn ** 3))
    Yp, _, _ = sph.sh_tables(n, np.array(1.0), np.array(0.0), np.array(1.0), np.array(0.0))
    y0 = complex(Yp[n][m])
    np.testing.assert_allclose(S, y0 / (2 * n + 1), atol=1e-12)
    np.testing.assert_allclose(D, -y0 / (2 * (2 * n + 1)), atol=1e-12)
    np.testing.assert_allclose(K, -y0 / (2 * (2 * n + 1)), atol=1e-12)


def test_exterior_expansions_match_upsampled_quadrature():
    """A density of degree 6 on the unit sphere: S^L, D^L and grad S^L at
    points 1.5 to 3 radii from the centre, by Eqs. 3.3-3.4 and by the smooth
    quadrature on a grid of order 48 (converged to rounding there)."""
    p = 6
    rng = np.random.default_rng(3)
    c = np.zeros((p + 1, p + 1), complex)
    for n in range(p + 1):
        c[n, 0] = rng.normal()
        c[n, 1:n + 1] = rng.normal(size=n) + 1j * rng.normal(size=n)
    P = 48
    x, nrm, w = quadrature.sphere_nodes(np.zeros(3), 1.0, P)
    ct, st, cp, sp, _ = sph.angles_of(x)
    q = laplace.synthesis(c, ct, st, cp, sp)
    d = rng.normal(size=(20, 3))
    xt = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(1.5, 3.0, size=(20, 1))
    np.testing.assert_allclose(laplace.ext_S(c, xt), laplace.sum_S(xt, x, q * w), atol=1e-12)
    np.testing.assert_allclose(laplace.ext_D(c, xt), laplace.sum_D(xt, x, nrm, q * w), atol=1e-12)
    np.testing.assert_allclose(laplace.ext_grad_S(c, xt), laplace.sum_grad(xt, x, q * w), atol=1e-12)
    # a target on the polar axis takes the rotated frame
    xa = np.array([[0.0, 0.0, 2.0], [1e-5, 0.0, -1.7]])
    np.testing.assert_allclose(laplace.ext_grad_S(c, xa), laplace.sum_grad(xa, x, q * w), atol=1e-12)


@pytest.mark.parametrize("eta,a", [(0.5, 1.0), (0.9, 0.7), (-0.3, 1.6)])
def test_permeable_sphere_in_uniform_field(eta, a):
    """q = 3 beta H0 . n with beta = 2 eta / (3 - eta) = (mu - mu0)/(mu + 2 mu0),
    whose exterior potential is the dipole beta a^3 H0 . x / r^3; the net
    magnetic force and torque on the sphere vanish."""
    H0 = np.array([0.3, -1.2, 0.8])
    c0 = np.array([0.5, 0.2, -0.1])
    g = ops.Geometry([c0], [a], 6)
    q, info = laplace.solve_magnetic(g, H0, eta, tol=1e-13)
    beta = 2 * eta / (3 - eta)
    np.testing.assert_allclose(q, 3 * beta * (g.nrm @ H0), atol=1e-12)
    coef = laplace.analysis(q, 6)
    xt = c0 + np.array([[2.0, 0.5, -0.3], [0.0, 0.0, 3.1]]) * a
    xh = (xt - c0) / a
    phi = a * laplace.ext_S(coef, xh)
    rr = np.linalg.norm(xt - c0, axis=1)
    np.testing.assert_allclose(phi, beta * a ** 3 * ((xt - c0) @ H0) / rr ** 3, atol=1e-12)
    f = laplace.maxwell_traction(g, q, H0)
    F, T = ops.moments(g, f)
    assert np.max(np.abs(F)) < 1e-11 and np.max(np.abs(T)) < 1e-11


@pytest.mark.parametrize("along", [True, False])
def test_two_spheres_far_apart_feel_the_dipole_force(along):
    """Induced dipoles m = 4 pi beta a^3 H0: along the field the spheres attract
    with 6 m^2 / (4 pi d^4); across it they repel with 3 m^2 / (4 pi d^4).  The
    relative deviation falls with the distance (induced-field corrections of
    relative size (a/d)^3)."""
    eta, a, H = 0.6, 1.0, 1.0
    beta = 2 * eta / (3 - eta)
    m = 4 * math.pi * beta * a ** 3 * H
    errs = []
    for d in (8.0, 16.0):
        e = np.array([0.0, 0.0, 1.0]) if along else np.array([1.0, 0.0, 0.0])
        g = ops.Geometry([np.zeros(3), d * e], [a, a], 6, eta=0.0)
        q, _ = laplace.solve_magnetic(g, [0.0, 0.0, H], eta, tol=1e-13)
        F, T = ops.moments(g, laplace.maxwell_traction(g, q, [0.0, 0.0, H]))
        ref = (-6.0 if along else 3.0) * m * m / (4 * math.pi * d ** 4)
        np.testing.assert_allclose(F[1], -F[0], atol=1e-9 * abs(ref))
        errs.append(abs(F[1] @ e - ref) / abs(ref))
    assert errs[1] < 0.02 and errs[1] < errs[0] / 4, errs


def test_mhd_mobility_depends_on_the_traction_only_through_its_moments():
    """With (1/2 I + K + L) mu = -(1/2 I + K) rho, tau = mu + rho solves
    (1/2 I + K + L) tau = L rho, which depends on rho only through its moments:
    the magnetic traction and the rigid-form density of the same force and
    torque give the same rigid motions.  Two spheres along the field attract
    (move towards each other, symmetrically)."""
    g = ops.Geometry([[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]], [1.0, 1.0], 6)
    F, T, v, w, info = osolve.solve_mhd(g, [0.0, 0.0, 2.0], 0.7, tol=1e-12)
    v2, w2, _ = osolve.solve_mobility(g, F, T, tol=1e-12)
    np.testing.assert_allclose(v, v2, atol=1e-10 * np.max(np.abs(v)))
    np.testing.assert_allclose(w, w2, atol=1e-10 * np.max(np.abs(v)))
    assert F[1][2] < 0 < F[0][2] and v[1][2] < 0 < v[0][2]
    np.testing.assert_allclose(v[0], -v[1], atol=1e-10)
