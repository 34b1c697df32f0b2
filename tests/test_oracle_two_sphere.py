"""The oracle's two-sphere resistance and mobility solves (Eqs. 5.8 and 5.19 with
the close-pair expansion of Sec. 4.2) against exact solutions for two equal
spheres that share nothing with the oracle: translation along the line of
centres in the same direction (Stimson-Jeffery) and towards each other
(Brenner), and rotation about it (Jeffery, both senses), checked against the
method of reflections; and far apart, Batchelor's (1976, J. Fluid Mech. 74,
1-29) expansions of the two-sphere mobility functions."""
import math

import numpy as np
import pytest

from classical import approach_lambda, jeffery_torque_ratio, stimson_jeffery_lambda
from oracle import operators as ops, solve


def test_series_matches_reflections_far_apart_and_contact_value():
    for d in (20.0, 40.0, 80.0):
        k = 1.0 / d
        assert abs(stimson_jeffery_lambda(d) - (1 - 1.5 * k + 2.25 * k * k)) <= 3.0 * k ** 3
    # the classical contact value (spheres touching: alpha -> 0)
    assert abs(stimson_jeffery_lambda(2.0 * math.cosh(1e-3)) - 0.645) < 1e-3


def _pair(d, p):
    return ops.Geometry([[0.1, -0.2, 0.3 - d / 2], [0.1, -0.2, 0.3 + d / 2]], [1.0, 1.0], p)


@pytest.mark.parametrize("d,tol", [(3.0, 2e-10), (2.5, 2e-9)])
def test_resistance_of_two_spheres_is_stimson_jeffery(d, tol):
    g = _pair(d, 12)
    U = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    F, T, _ = solve.solve_resistance(g, U, np.zeros((2, 3)), tol=1e-13)
    lam = stimson_jeffery_lambda(d)
    np.testing.assert_allclose(F[:, 2] / (6 * math.pi), lam, rtol=tol)
    np.testing.assert_allclose(F[:, :2], 0.0, atol=1e-12)
    np.testing.assert_allclose(T, 0.0, atol=1e-12)


def test_mobility_of_two_spheres_is_stimson_jeffery():
    d = 3.0
    g = _pair(d, 12)
    F = np.array([[0.0, 0.0, 6 * math.pi], [0.0, 0.0, 6 * math.pi]])
    v, w, _ = solve.solve_mobility(g, F, np.zeros((2, 3)), tol=1e-13)
    np.testing.assert_allclose(v[:, 2], 1.0 / stimson_jeffery_lambda(d), rtol=2e-10)
    np.testing.assert_allclose(v[:, :2], 0.0, atol=1e-12)
    np.testing.assert_allclose(w, 0.0, atol=1e-12)


def test_error_decays_spectrally_in_p():
    d = 3.0
    U = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    err = []
    for p in (6, 8, 10):
        F, _, _ = solve.solve_resistance(_pair(d, p), U, np.zeros((2, 3)), tol=1e-13)
        err.append(abs(F[0, 2] / (6 * math.pi) - stimson_jeffery_lambda(d)))
    assert err[1] < err[0] / 5 and err[2] < err[1] / 5


def test_torsion_series_match_rotlet_reflection_far_apart():
    for d in (10.0, 20.0):
        k = 1.0 / d
        assert abs(jeffery_torque_ratio(d, False) - (1 + k ** 3)) <= 2 * k ** 6
        assert abs(jeffery_torque_ratio(d, True) - (1 - k ** 3)) <= 2 * k ** 6


@pytest.mark.parametrize("co", [False, True])
def test_rotation_about_line_of_centres_is_jeffery(co):
    d = 3.0
    g = _pair(d, 12)
    W = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0 if co else -1.0]])
    F, T, _ = solve.solve_resistance(g, np.zeros((2, 3)), W, tol=1e-13)
    np.testing.assert_allclose(T[:, 2] / (8 * math.pi * W[:, 2]), jeffery_torque_ratio(d, co), rtol=1e-10)
    np.testing.assert_allclose(T[:, :2], 0.0, atol=1e-12)
    np.testing.assert_allclose(F, 0.0, atol=1e-12)
    # the inverse problem: torques given, angular velocities follow
    v, w, _ = solve.solve_mobility(g, np.zeros((2, 3)), 8 * math.pi * W, tol=1e-13)
    np.testing.assert_allclose(w[:, 2] / W[:, 2], 1.0 / jeffery_torque_ratio(d, co), rtol=1e-10)
    np.testing.assert_allclose(v, 0.0, atol=1e-12)


def test_approach_series_matches_reflections_far_apart():
    for d in (20.0, 40.0, 80.0):
        k = 1.0 / d
        assert abs(approach_lambda(d) - (1 + 1.5 * k + 2.25 * k * k)) <= 3.0 * k ** 3


@pytest.mark.parametrize("d,p,tol", [(3.0, 12, 2e-9), (2.5, 14, 1e-7)])
def test_spheres_approaching_each_other_is_brenner(d, p, tol):
    g = _pair(d, p)
    U = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    F, T, _ = solve.solve_resistance(g, U, np.zeros((2, 3)), tol=1e-13)
    np.testing.assert_allclose(F[:, 2] / (6 * math.pi * U[:, 2]), approach_lambda(d), rtol=tol)
    np.testing.assert_allclose(F[:, :2], 0.0, atol=1e-11)
    np.testing.assert_allclose(T, 0.0, atol=1e-11)


@pytest.mark.parametrize("r", [10.0, 20.0])
def test_far_apart_mobilities_follow_batchelor_expansions(r):
    """A force on sphere 1 only, along and across the line of centres, in units
    of F / (6 pi a): x11 = 1 - 15/(4 r^4), x12 = 3/(2r) - 1/r^3, y11 =
    1 - 17/(16 r^6), y12 = 3/(4r) + 1/(2 r^3) (r = d / a), each up to its next
    order; sphere 2 turns with the Stokeslet's vorticity, -3/(4 r^2)."""
    g = _pair(r, 8)
    F = np.zeros((2, 3))
    F[0, 2] = 6 * math.pi
    v, w, _ = solve.solve_mobility(g, F, np.zeros((2, 3)), tol=1e-13)
    assert abs(v[0, 2] - (1 - 15 / (4 * r ** 4))) <= 8 / r ** 6
    assert abs(v[1, 2] - (1.5 / r - 1 / r ** 3)) <= 25 / r ** 7
    np.testing.assert_allclose(w, 0.0, atol=1e-12)
    F = np.zeros((2, 3))
    F[0, 0] = 6 * math.pi
    v, w, _ = solve.solve_mobility(g, F, np.zeros((2, 3)), tol=1e-13)
    assert abs(v[0, 0] - (1 - 17 / (16 * r ** 6))) <= 4 / r ** 8
    assert abs(v[1, 0] - (0.75 / r + 0.5 / r ** 3)) <= 1 / r ** 9
    assert abs(w[1, 1] + 0.75 / r ** 2) <= 1 / r ** 8
