"""The CUDA path against exact solutions for two equal spheres, independent of the
oracle: translation along the line of centres in the same direction
(Stimson-Jeffery) and towards each other (Brenner), rotation about it (Jeffery),
and far apart Batchelor's mobility expansions; resistance and mobility in FP64,
double-float and mixed precision, and mixed precision with the exact pair
preconditioner."""
import math

import numpy as np
import pytest

from classical import approach_lambda, jeffery_torque_ratio, stimson_jeffery_lambda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def _centres(d):
    return np.array([[0.1, -0.2, 0.3 - d / 2], [0.1, -0.2, 0.3 + d / 2]])


@pytest.mark.parametrize("prec,precond", [(0, 0), (2, 0), (1, 0), (1, 2)])
def test_resistance_of_two_spheres_is_stimson_jeffery(sb, prec, precond):
    d = 3.0
    U = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    with sb.SphereBIE(_centres(d), np.ones(2), 12, prec=prec, tol=1e-11, precond=precond) as s:
        F, T, info = s.resistance(U, np.zeros((2, 3)))
    assert info["status"] == 0
    np.testing.assert_allclose(F[:, 2] / (6 * math.pi), stimson_jeffery_lambda(d), rtol=1e-9)
    np.testing.assert_allclose(F[:, :2], 0.0, atol=1e-9)
    np.testing.assert_allclose(T, 0.0, atol=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_mobility_of_two_spheres_is_stimson_jeffery(sb, prec):
    d = 2.5
    F = np.array([[0.0, 0.0, 6 * math.pi], [0.0, 0.0, 6 * math.pi]])
    with sb.SphereBIE(_centres(d), np.ones(2), 12, prec=prec, tol=1e-11) as s:
        v, w, info = s.mobility(F, np.zeros((2, 3)))
    assert info["status"] == 0
    np.testing.assert_allclose(v[:, 2], 1.0 / stimson_jeffery_lambda(d), rtol=1e-8)
    np.testing.assert_allclose(v[:, :2], 0.0, atol=1e-9)
    np.testing.assert_allclose(w, 0.0, atol=1e-9)


@pytest.mark.parametrize("prec,co", [(0, False), (1, True), (2, False)])
def test_rotation_about_line_of_centres_is_jeffery(sb, prec, co):
    d = 3.0
    W = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0 if co else -1.0]])
    with sb.SphereBIE(_centres(d), np.ones(2), 12, prec=prec, tol=1e-11) as s:
        F, T, info = s.resistance(np.zeros((2, 3)), W)
        v, w, info2 = s.mobility(np.zeros((2, 3)), 8 * math.pi * W)
    assert info["status"] == 0 and info2["status"] == 0
    ratio = jeffery_torque_ratio(d, co)
    np.testing.assert_allclose(T[:, 2] / (8 * math.pi * W[:, 2]), ratio, rtol=1e-9)
    np.testing.assert_allclose(w[:, 2] / W[:, 2], 1.0 / ratio, rtol=1e-9)
    np.testing.assert_allclose(F, 0.0, atol=1e-9)
    np.testing.assert_allclose(v, 0.0, atol=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_spheres_approaching_each_other_is_brenner(sb, prec):
    d = 3.0
    U = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    with sb.SphereBIE(_centres(d), np.ones(2), 12, prec=prec, tol=1e-11) as s:
        F, T, info = s.resistance(U, np.zeros((2, 3)))
    assert info["status"] == 0
    np.testing.assert_allclose(F[:, 2] / (6 * math.pi * U[:, 2]), approach_lambda(d), rtol=3e-9)
    np.testing.assert_allclose(T, 0.0, atol=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_far_apart_mobilities_follow_batchelor_expansions(sb, prec):
    r = 10.0
    F = np.zeros((2, 3))
    F[0, 2] = F[1, 0] = 6 * math.pi  # sphere 1 along the line, sphere 2 across it
    with sb.SphereBIE(_centres(r), np.ones(2), 8, prec=prec, tol=1e-11) as s:
        v, w, info = s.mobility(F, np.zeros((2, 3)))
    assert info["status"] == 0
    # by linearity: sphere 1 gets x11 along and y12 across; sphere 2 gets x12 along and y11 across
    assert abs(v[0, 2] - (1 - 15 / (4 * r ** 4))) <= 8 / r ** 6
    assert abs(v[1, 2] - (1.5 / r - 1 / r ** 3)) <= 25 / r ** 7
    assert abs(v[1, 0] - (1 - 17 / (16 * r ** 6))) <= 4 / r ** 8
    assert abs(v[0, 0] - (0.75 / r + 0.5 / r ** 3)) <= 1 / r ** 9
