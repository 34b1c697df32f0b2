"""Pins of the oracle's grid, quadrature and spherical harmonics against
library routines and closed forms (Sec. 2.1, Eqs. 2.1-2.6; Sec. 4, Eqs. 4.2-4.4)."""
import math

import numpy as np
import pytest
import scipy.special as sps

from oracle import quadrature, sph, vsh


@pytest.mark.parametrize("n", [1, 2, 3, 7, 13, 25])
def test_gauss_legendre_matches_numpy(n):
    t, lam = quadrature.gauss_legendre(n)
    tn, ln = np.polynomial.legendre.leggauss(n)
    assert np.all(np.diff(t) < 0)
    np.testing.assert_allclose(t[::-1], tn, atol=2e-15)
    np.testing.assert_allclose(lam[::-1], ln, atol=2e-15)


@pytest.mark.parametrize("n", [3, 8, 13])
def test_gauss_legendre_exact_monomials(n):
    t, lam = quadrature.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(lam * t ** k) - exact) < 1e-14


def test_sphere_weights_area_and_moments():
    for a in (0.5, 1.0, 2.0):
        x, nr, w = quadrature.sphere_nodes([0.3, -1.0, 2.0], a, 7)
        assert abs(w.sum() - 4 * math.pi * a * a) < 1e-12 * a * a
        # int (x - c)(x - c)^T = (4 pi a^4 / 3) I
        d = x - np.array([0.3, -1.0, 2.0])
        np.testing.assert_allclose((w[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0),
                                   4 * math.pi * a ** 4 / 3 * np.eye(3), atol=1e-12 * a ** 4)
        np.testing.assert_allclose(np.linalg.norm(nr, axis=1), 1.0, atol=1e-15)


def test_legendre_Q_matches_numpy_derivatives():
    t = np.linspace(-0.99, 0.99, 17)
    Q = sph.legendre_Q(9, t)
    for n in range(10):
        coef = np.zeros(n + 1)
        coef[n] = 1.0
        for m in range(n + 1):
            ref = np.polynomial.legendre.legval(t, np.polynomial.legendre.legder(coef, m)) if m else \
                np.polynomial.legendre.legval(t, coef)
            np.testing.assert_allclose(Q[n][m], ref, rtol=1e-12, atol=1e-12 * abs(ref).max())


def test_Y_matches_scipy_without_condon_shortley():
    rng = np.random.default_rng(0)
    th = rng.uniform(0, np.pi, 11)
    ph = rng.uniform(0, 2 * np.pi, 11)
    Y, dY, mY = sph.sh_tables(8, np.cos(th), np.sin(th), np.cos(ph), np.sin(ph))
    for n in range(9):
        for m in range(n + 1):
            ref = (-1) ** m * sps.sph_harm_y(n, m, th, ph)
            np.testing.assert_allclose(Y[n][m], ref, rtol=1e-12, atol=1e-13)


def test_dY_dtheta_and_mY_by_finite_differences():
    rng = np.random.default_rng(1)
    th = rng.uniform(0.1, np.pi - 0.1, 7)
    ph = rng.uniform(0, 2 * np.pi, 7)
    h = 1e-5
    f = lambda a, b: sph.sh_tables(6, np.cos(a), np.sin(a), np.cos(b), np.sin(b))[0]
    Y, dY, mY = sph.sh_tables(6, np.cos(th), np.sin(th), np.cos(ph), np.sin(ph))
    Yp, Ym = f(th + h, ph), f(th - h, ph)
    Pp, Pm = f(th, ph + h), f(th, ph - h)
    for n in range(7):
        for m in range(n + 1):
            np.testing.assert_allclose(dY[n][m], (Yp[n][m] - Ym[n][m]) / (2 * h), atol=1e-8)
            np.testing.assert_allclose(mY[n][m], (Pp[n][m] - Pm[n][m]) / (2 * h) / np.sin(th), atol=1e-8)


@pytest.mark.parametrize("p", [2, 5, 9])
def test_discrete_orthonormality(p):
    ct, st, cp, sp = vsh.grid_angles(p)
    w = quadrature.unit_weights(p)
    Y, V, W, X = sph.vsh_tables(p, ct, st, cp, sp)
    idx = [(n, m) for n in range(p + 1) for m in range(n + 1)]
    for (n, m) in idx:
        for (k, l) in idx:
            g = np.sum(w * Y[n][m] * np.conj(Y[k][l]))
            assert abs(g - (1.0 if (n, m) == (k, l) else 0.0)) < 1e-13
    # VSH norms and orthogonality: |V|^2 = (n+1)(2n+1), |W|^2 = n(2n+1), |X|^2 = n(n+1)
    ip = lambda A, B: np.sum(w * sum(A[i] * np.conj(B[i]) for i in range(3)))
    for n in range(1, p + 1):
        for m in range(n + 1):
            assert abs(ip(V[n][m], V[n][m]) - (n + 1) * (2 * n + 1)) < 1e-11 * n * n
            assert abs(ip(W[n][m], W[n][m]) - n * (2 * n + 1)) < 1e-11 * n * n
            assert abs(ip(X[n][m], X[n][m]) - n * (n + 1)) < 1e-11 * n * n
            assert abs(ip(V[n][m], W[n][m])) < 1e-11 * n * n
            assert abs(ip(V[n][m], X[n][m])) < 1e-11 * n * n
            assert abs(ip(W[n][m], X[n][m])) < 1e-11 * n * n


def test_rigid_fields_are_W1_and_X1():
    """A constant field is W_1 and a rotation is X_1 (used by the null-space
    statements of Eq. 5.8): e_z = W_1[cos] and e_z x e_r = -X_1[cos]."""
    p = 4
    ct, st, cp, sp = vsh.grid_angles(p)
    n_nodes = ct.size
    F = np.tile([0.0, 0.0, 1.0], (n_nodes, 1))
    c = vsh.analysis(F, p)
    y10 = math.sqrt(3.0 / (4 * math.pi))
    expect = np.zeros_like(c)
    expect[1, 1, 0] = 1.0 / y10
    np.testing.assert_allclose(c, expect, atol=1e-13)
    er = np.stack([st * cp, st * sp, ct], -1).reshape(-1, 3)
    R = np.cross([0.0, 0.0, 1.0], er)
    c = vsh.analysis(R, p)
    expect = np.zeros_like(c)
    expect[2, 1, 0] = -1.0 / y10
    np.testing.assert_allclose(c, expect, atol=1e-13)


def _random_coeffs(rng, p):
    c = rng.normal(size=(3, p + 1, p + 1)) + 1j * rng.normal(size=(3, p + 1, p + 1))
    for n in range(p + 1):
        c[:, n, n + 1:] = 0
    c[:, :, 0] = c[:, :, 0].real
    c[1, 0, 0] = 0
    c[2, 0, 0] = 0
    return c


@pytest.mark.parametrize("p", [1, 2, 5, 8, 24])  # 24: the largest order the library accepts
def test_analysis_inverts_synthesis(p):
    rng = np.random.default_rng(p)
    c = _random_coeffs(rng, p)
    np.testing.assert_allclose(vsh.analysis(vsh.synthesis(c), p), c, atol=1e-12)


def test_synthesis_on_finer_grid_is_band_limited_interpolation():
    rng = np.random.default_rng(7)
    c = _random_coeffs(rng, 4)
    fine = vsh.synthesis(c, p_out=9)
    c9 = vsh.analysis(fine, 9)
    np.testing.assert_allclose(c9[:, :5, :5], c, atol=1e-12)
    assert np.max(np.abs(c9[:, 5:, :])) < 1e-12
