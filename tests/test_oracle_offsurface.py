"""Pins of the exterior formulas (Eqs. 3.6-3.11) and the traction of the
single layer (Eq. 3.18) against upsampled smooth quadrature (Eq. 4.4) of the
kernels (Eqs. 2.19-2.22), the Stokes equations (Eq. 5.1) by finite
differences, and the Stokeslet pressure."""
import math

import numpy as np
import pytest

from oracle import kernels, offsurface, quadrature, signatures, vsh


def _coeffs(rng, p):
    c = rng.normal(size=(3, p + 1, p + 1)) + 1j * rng.normal(size=(3, p + 1, p + 1))
    for n in range(p + 1):
        c[:, n, n + 1:] = 0
    c[:, :, 0] = c[:, :, 0].real
    c[1, 0, 0] = 0
    c[2, 0, 0] = 0
    return c


def _upsampled(c, pu=40):
    p = c.shape[1] - 1
    xs, ns, ws = quadrature.sphere_nodes([0, 0, 0], 1.0, pu)
    cu = np.zeros((3, pu + 1, pu + 1), complex)
    cu[:, :p + 1, :p + 1] = c
    return xs, ns, ws, vsh.synthesis(cu)


def _targets(rng, m, rmin=1.5, rmax=3.0):
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    nt = rng.normal(size=(m, 3))
    nt /= np.linalg.norm(nt, axis=1)[:, None]
    return d * rng.uniform(rmin, rmax, size=(m, 1)), nt


@pytest.mark.parametrize("p", [2, 4])
def test_exterior_formulas_match_upsampled_quadrature(p):
    rng = np.random.default_rng(10 + p)
    c = _coeffs(rng, p)
    xs, ns, ws, sig = _upsampled(c)
    xt, nt = _targets(rng, 25)
    dw = sig * ws[:, None]
    for got, ref in ((offsurface.S_velocity(c, xt), kernels.stokeslet_sum(xt, xs, dw)),
                     (offsurface.D_velocity(c, xt), kernels.stresslet_sum_D(xt, xs, ns, dw)),
                     (offsurface.S_traction(c, xt, nt), kernels.stresslet_sum_K(xt, nt, xs, dw))):
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_traction_near_polar_axis_uses_rotated_frame():
    rng = np.random.default_rng(3)
    c = _coeffs(rng, 4)
    xs, ns, ws, sig = _upsampled(c)
    xt = np.array([[1e-7, 2e-7, 1.7], [0, 0, -2.0], [3e-4, 0, 1.6], [2e-3, 1e-3, -1.9], [0.5, 0.4, 1.6]])
    nt = rng.normal(size=xt.shape)
    nt /= np.linalg.norm(nt, axis=1)[:, None]
    ref = kernels.stresslet_sum_K(xt, nt, xs, sig * ws[:, None])
    got = offsurface.S_traction(c, xt, nt)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_surface_limits_reproduce_signatures():
    """At r = 1 the exterior branches give S and D+ of Theorem 2 (Eqs. 3.6-3.12),
    and the traction with n = e_r gives K+ (Eqs. 3.19-3.21)."""
    rng = np.random.default_rng(5)
    p = 5
    c = _coeffs(rng, p)
    ct, st, cp, sp = vsh.grid_angles(p)
    er = np.stack([st * cp, st * sp, ct], -1).reshape(-1, 3)
    for table, got in ((signatures.S, offsurface.S_velocity(c, er)),
                       (signatures.D_plus, offsurface.D_velocity(c, er)),
                       (signatures.K_plus, offsurface.S_traction(c, er * (1 + 1e-13), er))):
        cl = c.copy()
        for n in range(p + 1):
            for t in range(3):
                cl[t, n] *= table(n)[t]
        cl[1, 0, 0] = 0
        cl[2, 0, 0] = 0
        np.testing.assert_allclose(got, vsh.synthesis(cl), atol=1e-9)


def test_exterior_single_layer_solves_stokes():
    """-Lap u + grad p = 0 and div u = 0 (Eq. 5.1) for the exterior S expansion
    with the pressure of Sec. 3.2, by 4th-order central differences."""
    rng = np.random.default_rng(9)
    c = _coeffs(rng, 4)
    x0, _ = _targets(rng, 6, 1.6, 2.5)
    h = 2e-3
    f = lambda x: offsurface.S_velocity(c, x)
    g = lambda x: offsurface.S_pressure(c, x)
    def d1(fun, x, i):
        e = np.zeros(3)
        e[i] = h
        return (-fun(x + 2 * e) + 8 * fun(x + e) - 8 * fun(x - e) + fun(x - 2 * e)) / (12 * h)
    def d2(fun, x, i):
        e = np.zeros(3)
        e[i] = h
        return (-fun(x + 2 * e) + 16 * fun(x + e) - 30 * fun(x) + 16 * fun(x - e) - fun(x - 2 * e)) / (12 * h * h)
    lap = sum(d2(f, x0, i) for i in range(3))
    gp = np.stack([d1(g, x0, i) for i in range(3)], -1)
    div = sum(d1(f, x0, i)[:, i] for i in range(3))
    scale = np.max(np.abs(lap))
    assert np.max(np.abs(-lap + gp)) < 1e-6 * scale
    assert np.max(np.abs(div)) < 1e-8 * np.max(np.abs(f(x0)))


def test_exterior_double_layer_is_divergence_free():
    rng = np.random.default_rng(11)
    c = _coeffs(rng, 4)
    x0, _ = _targets(rng, 6, 1.6, 2.5)
    h = 2e-3
    div = 0.0
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        f = lambda x: offsurface.D_velocity(c, x)[:, i]
        div = div + (-f(x0 + 2 * e) + 8 * f(x0 + e) - 8 * f(x0 - e) + f(x0 - 2 * e)) / (12 * h)
    assert np.max(np.abs(div)) < 1e-8 * np.max(np.abs(offsurface.D_velocity(c, x0)))


def test_single_layer_pressure_is_stokeslet_pressure():
    """A uniform density f on the unit sphere has total force 4 pi f; outside,
    its pressure is exactly the Stokeslet pressure (r . F) / (4 pi r^3)."""
    f = np.array([0.3, -0.5, 0.8])
    p = 3
    ct, st, cp, sp = vsh.grid_angles(p)
    c = vsh.analysis(np.tile(f, (ct.size, 1)), p)
    rng = np.random.default_rng(2)
    x, _ = _targets(rng, 10, 1.2, 4.0)
    F = 4 * math.pi * f
    ref = x @ F / (4 * math.pi * np.linalg.norm(x, axis=1) ** 3)
    np.testing.assert_allclose(offsurface.S_pressure(c, x), ref, atol=1e-13)
