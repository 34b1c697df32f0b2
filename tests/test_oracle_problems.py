"""Pins of the oracle's porous-media (Problem 1, Eq. 5.4) and squirmer
(Problem 4, Eqs. 5.14-5.17) drivers against what fixes them independently:
Stokes drag and the Faxen torque of one fixed sphere, the resistance problem's
completed double layer (Eq. 5.19) -- a different integral equation for the
same flow -- on suspensions with close pairs, the swimming speed 2 B1 / 3 of a
single squirmer (Lighthill, Blake), the force- and torque-free motion that a
rigid slip field must produce, and a resistance-matrix solution of the
squirmer problem (Eq. 5.19 again), each converging spectrally in p."""
import math

import numpy as np
import pytest

from oracle import operators as ops
from oracle import solve as osolve
from paper_1707_06551_gb300 import workloads as wl


@pytest.mark.parametrize("a", [0.5, 2.0])
def test_porous_single_sphere_stokes_drag(a):
    """A fixed sphere in a uniform stream U exerts -6 pi a U on the fluid."""
    g = ops.Geometry([[0.3, -0.2, 0.1]], [a], 6)
    U = np.array([0.7, -0.4, 1.1])
    F, T, info = osolve.solve_porous(g, u0=U, tol=1e-13)
    np.testing.assert_allclose(F[0], -6 * math.pi * a * U, rtol=1e-10)
    assert np.max(np.abs(T)) < 1e-10 * a ** 3


def test_porous_single_sphere_faxen_torque():
    """A fixed sphere at the origin of the shear u = (y, 0, 0): no force; the
    torque it exerts on the fluid is -8 pi a^3 Omega_inf with
    Omega_inf = curl(u)/2 = (0, 0, -1/2)."""
    a = 1.3
    g = ops.Geometry([[0.0, 0.0, 0.0]], [a], 6)
    G = np.zeros((3, 3))
    G[0, 1] = 1.0
    F, T, _ = osolve.solve_porous(g, G=G, tol=1e-13)
    assert np.max(np.abs(F)) < 1e-10
    np.testing.assert_allclose(T[0], [0.0, 0.0, 4 * math.pi * a ** 3], atol=1e-10)


def test_porous_agrees_with_completed_double_layer():
    """Fixed spheres in a random linear flow: the porous-media equation
    (1/2 I + S + D) mu = -u_inf and the resistance equation
    (1/2 I + D + N) psi = -u_inf describe the same Stokes flow, so their forces
    and torques agree up to the discretisation error, which falls
    geometrically with p."""
    w = wl.small_suspension(4, 4, seed=8, radius_range=(0.8, 1.2), gap_range=(0.3, 0.5))
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=3)
    G = rng.normal(size=(3, 3))
    G -= np.trace(G) / 3 * np.eye(3)
    errs = []
    for p in (4, 6, 8, 10):
        g = ops.Geometry(w["centres"], w["radii"], p)
        Fp, Tp, _ = osolve.solve_porous(g, u0, G, tol=1e-13)
        Fr, Tr, _ = osolve.solve_resistance(g, np.zeros((g.n, 3)), np.zeros((g.n, 3)), u0, G, tol=1e-13)
        errs.append(max(np.max(np.abs(Fp - Fr)) / np.max(np.abs(Fr)), np.max(np.abs(Tp - Tr)) / np.max(np.abs(Tr))))
    assert errs[-1] < 1e-6, errs
    assert errs[0] > 10 * errs[-1], errs
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs


def _slip(g, axes, B1, B2):
    ax = np.repeat(np.asarray(axes, float).reshape(-1, 3), g.npn, axis=0)
    return wl.squirmer_slip(g.nrm, ax, B1, B2)


@pytest.mark.parametrize("B2", [0.0, -3.0, 5.0])
def test_single_squirmer_swims_at_two_thirds_B1(B2):
    """u_s = (B1 + B2 cos t) sin t e_t on a free sphere: it translates along
    its axis at 2 B1 / 3 whatever B2, without rotating."""
    a, B1 = 1.4, 0.8
    e = np.array([0.3, -0.5, 0.8])
    e /= np.linalg.norm(e)
    g = ops.Geometry([[0.2, 0.1, -0.3]], [a], 8)
    v, om, info = osolve.solve_squirmer(g, _slip(g, [e], B1, B2), tol=1e-13)
    np.testing.assert_allclose(v[0], 2.0 / 3.0 * B1 * e, atol=1e-10)
    assert np.max(np.abs(om)) < 1e-10
    dens = info["density"]
    M0, M1 = ops.moments(g, dens)
    assert np.max(np.abs(M0)) < 1e-10 and np.max(np.abs(M1)) < 1e-10


def test_rigid_slip_is_cancelled_by_the_rigid_motion():
    """A slip field that is itself a rigid motion V_i + W_i x (x - c_i) leaves
    force- and torque-free spheres moving with -V_i, -W_i (the flow is zero),
    with close pairs present."""
    w = wl.small_suspension(4, 6, seed=12, radius_range=(0.7, 1.3))
    g = ops.Geometry(w["centres"], w["radii"], 6)
    rng = np.random.default_rng(5)
    V, W = rng.normal(size=(g.n, 3)), rng.normal(size=(g.n, 3))
    slip = np.zeros((g.N, 3))
    for k in range(g.n):
        s = g.sl(k)
        slip[s] = V[k] + np.cross(W[k], g.x[s] - g.c[k])
    v, om, info = osolve.solve_squirmer(g, slip, tol=1e-13)
    np.testing.assert_allclose(v, -V, atol=1e-9)
    np.testing.assert_allclose(om, -W, atol=1e-9)
    assert np.max(np.abs(info["density"])) < 1e-9


def _squirmer_by_resistance(g, slip):
    """Force- and torque-free velocities from the resistance problem: with
    boundary velocity v + w x r + u_s the forces are R (v, w) + F_s, R and F_s
    from completed-double-layer solves; setting them to zero gives (v, w)."""
    n = g.n
    R = np.zeros((6 * n, 6 * n))
    for j in range(6 * n):
        e = np.zeros(6 * n)
        e[j] = 1.0
        F, T, _ = osolve.solve_resistance(g, e[:3 * n].reshape(n, 3), e[3 * n:].reshape(n, 3), tol=1e-13)
        R[:, j] = np.concatenate([F.ravel(), T.ravel()])
    F, T, _ = osolve.solve_resistance(g, None, None, tol=1e-13, rhs=slip)
    vw = np.linalg.solve(R, -np.concatenate([F.ravel(), T.ravel()]))
    return vw[:3 * n].reshape(n, 3), vw[3 * n:].reshape(n, 3)


def test_squirmers_agree_with_resistance_matrix_solution():
    """Three pusher squirmers with close pairs: the square form of Eq. 5.17
    and the resistance-matrix route give the same velocities up to the
    discretisation error, which falls with p."""
    w = wl.squirmers(3, 4, seed=21, beta=-3.0, radius_range=(0.8, 1.2))
    errs = []
    for p in (4, 6, 8):
        g = ops.Geometry(w["centres"], w["radii"], p)
        slip = _slip(g, w["axes"], w["B1"], w["B2"])
        v, om, _ = osolve.solve_squirmer(g, slip, tol=1e-13)
        vr, wr = _squirmer_by_resistance(g, slip)
        scale = max(np.max(np.abs(vr)), np.max(np.abs(wr)))
        errs.append(max(np.max(np.abs(v - vr)), np.max(np.abs(om - wr))) / scale)
    assert errs[-1] < 1e-5, errs
    assert errs[0] > 10 * errs[-1], errs
