"""Pins of the oracle's discrete operators and solves (Sec. 4-6) against
closed forms (Stokes drag and rotational torque, Faxen's laws, the double-layer
jump on constants), a manufactured solution (Sec. 6, Eq. 6.2), reciprocity of
mobility and resistance, and a dense library solve."""
import math

import numpy as np
import pytest

from oracle import gmres, kernels, operators as ops, solve


@pytest.mark.parametrize("a", [0.5, 2.0])
def test_single_sphere_drag_and_torque(a):
    g = ops.Geometry([[0.3, -0.2, 0.1]], [a], 6)
    U = np.array([[1.0, 0.5, -0.3]])
    W = np.array([[0.2, -0.7, 0.4]])
    F, T, _ = solve.solve_resistance(g, U, np.zeros((1, 3)), tol=1e-13)
    np.testing.assert_allclose(F, 6 * math.pi * a * U, rtol=1e-11)
    np.testing.assert_allclose(T, 0.0, atol=1e-11)
    F, T, _ = solve.solve_resistance(g, np.zeros((1, 3)), W, tol=1e-13)
    np.testing.assert_allclose(T, 8 * math.pi * a ** 3 * W, rtol=1e-11)
    np.testing.assert_allclose(F, 0.0, atol=1e-11)
    v, w, info = solve.solve_mobility(g, 6 * math.pi * a * U, 8 * math.pi * a ** 3 * W, tol=1e-13)
    np.testing.assert_allclose(v, U, rtol=1e-11)
    np.testing.assert_allclose(w, W, rtol=1e-11)


def test_double_layer_of_constant_density():
    """D[c] = -c inside, 0 outside, principal value -c/2 on the surface."""
    g = ops.Geometry([[0, 0, 0], [5.0, 0.5, 0.0]], [1.0, 0.7], 6, eta=1.0)
    c = np.array([0.4, -1.1, 0.25])
    dens = np.zeros((g.N, 3))
    dens[g.sl(0)] = c
    out = ops.layer(g, "D", dens)
    np.testing.assert_allclose(out[g.sl(0)], -0.5 * np.tile(c, (g.npn, 1)), atol=1e-13)
    np.testing.assert_allclose(out[g.sl(1)], 0.0, atol=1e-7)


def test_faxen_fixed_sphere_in_shear():
    """A fixed sphere at the origin in u_inf = (y, 0, 0): no force; the torque
    it exerts on the fluid is -8 pi a^3 Omega_inf with Omega_inf = (0, 0, -1/2)."""
    a = 0.8
    g = ops.Geometry([[0.0, 0.0, 0.0]], [a], 5)
    G = np.zeros((3, 3))
    G[0, 1] = 1.0
    F, T, _ = solve.solve_resistance(g, np.zeros((1, 3)), np.zeros((1, 3)), G=G, tol=1e-13)
    np.testing.assert_allclose(F, 0.0, atol=1e-11)
    np.testing.assert_allclose(T[0], [0.0, 0.0, 4 * math.pi * a ** 3], atol=1e-11)


@pytest.mark.parametrize("op", ["S", "D", "K"])
def test_near_expansion_agrees_with_quadrature_when_separated(op):
    """For well-separated spheres the exterior expansion (near path) and the
    smooth quadrature (far path) approximate the same integral; their gap
    falls geometrically with p."""
    cen = [[0, 0, 0], [4.2, 1.0, -0.5], [-1.0, 4.5, 1.0]]
    rad = [1.0, 0.8, 1.2]
    errs = []
    for p in (8, 16):
        rng = np.random.default_rng(4)
        g_far = ops.Geometry(cen, rad, p, eta=0.0)
        g_near = ops.Geometry(cen, rad, p, eta=10.0)
        assert g_far.n_near_pairs() == 0 and g_near.n_near_pairs() == 6
        dens = rng.normal(size=(g_far.N, 3))
        a = ops.layer(g_far, op, dens)
        b = ops.layer(g_near, op, dens)
        errs.append(np.max(np.abs(a - b)) / np.max(np.abs(a)))
    assert errs[1] < errs[0] / 100 and errs[1] < 2e-7


E2_RADII = np.array([0.903, 0.510, 0.262])
E2_CENTRES = np.array([[0.0, 0.0, 0.0], [1.70, 0.35, 0.20], [0.40, 1.35, -0.45]])


def _manufactured(p):
    rng = np.random.default_rng(21)
    g = ops.Geometry(E2_CENTRES, E2_RADII, p, eta=1.0)
    dirs = rng.normal(size=(3, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    src = E2_CENTRES + 0.5 * E2_RADII[:, None] * dirs
    f = rng.normal(size=(3, 3))
    b = sum(kernels.stokeslet(g.x, src[l], f[l]) for l in range(3))
    F, T, info = solve.solve_resistance(g, None, None, rhs=b, tol=1e-12)
    errF = np.max(np.abs(F - f))
    errT = np.max(np.abs(T - np.cross(src - E2_CENTRES, f)))
    return errF, errT, g


def test_manufactured_resistance_converges_spectrally():
    """Stokeslets f_l inside each sphere (Sec. 6, Eq. 6.2): the completed double
    layer returns int psi = f_l and int (y - c_l) x psi = (p_l - c_l) x f_l,
    with errors falling geometrically in p."""
    errs = []
    for p in (4, 8, 12):
        eF, eT, g = _manufactured(p)
        assert g.n_near_pairs() > 0
        errs.append(max(eF, eT))
    assert errs[0] > 100 * errs[1] and errs[1] > 10 * errs[2]
    assert errs[2] < 5e-6


def test_reciprocity_mobility_resistance():
    """Mobility of the forces a resistance solve returns gives back the imposed
    rigid motions (two independent formulations, Eqs. 5.8 and 5.19); the gap
    closes geometrically in p."""
    cen = np.array([[0, 0, 0], [2.3, 0.2, 0.1], [0.5, -2.4, 0.3]])
    errs = []
    for p in (6, 10):
        rng = np.random.default_rng(8)
        g = ops.Geometry(cen, [1.0, 1.0, 1.0], p)
        assert g.n_near_pairs() == 6
        v = rng.normal(size=(3, 3))
        w = rng.normal(size=(3, 3))
        F, T, _ = solve.solve_resistance(g, v, w, tol=1e-12)
        v2, w2, _ = solve.solve_mobility(g, F, T, tol=1e-12)
        errs.append(max(np.max(np.abs(v2 - v)), np.max(np.abs(w2 - w))))
    assert errs[1] < errs[0] / 50 and errs[1] < 1e-5


def test_gmres_matches_dense_solve():
    g = ops.Geometry([[0, 0, 0], [2.4, 0.3, 0.0]], [1.0, 0.9], 2)
    n = 3 * g.N
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = ops.apply(g, "resistance", e.reshape(-1, 3)).ravel()
    rng = np.random.default_rng(0)
    b = rng.normal(size=n)
    x_ref = np.linalg.solve(A, b)
    x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-13)
    assert info["converged"]
    assert np.max(np.abs(x - x_ref)) < 1e-10 * np.max(np.abs(x_ref))
    x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-13, restart=7)
    assert info["converged"]
    assert np.max(np.abs(x - x_ref)) < 1e-10 * np.max(np.abs(x_ref))


def test_overlap_rejected():
    with pytest.raises(ops.OverlapError):
        ops.Geometry([[0, 0, 0], [1.9, 0, 0]], [1.0, 1.0], 4)
