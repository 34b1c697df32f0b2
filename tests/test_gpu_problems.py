"""The porous-media (Problem 1, Eq. 5.4) and squirmer (Problem 4, Eqs.
5.14-5.17) problems on the CUDA path: operator applies against the oracle
(FP64 and double-float: 1e-10; mixed precision: 2e-5, per sphere), solves
against oracle solves, the closed forms the oracle is pinned to (drag, the
squirmer's 2 B1 / 3), and a batch of problems against separate contexts."""
import math

import numpy as np
import pytest

from oracle import operators as ops
from oracle import solve as osolve
from paper_1707_06551_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def _per_sphere(got, ref, npn):
    return np.max(np.abs(got - ref).reshape(-1, npn, 3), axis=(1, 2)) / np.max(
        np.abs(ref).reshape(-1, npn, 3), axis=(1, 2))


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (2, TOL64), (1, TOL32)])
@pytest.mark.parametrize("op", ["porous", "squirmer"])
@pytest.mark.parametrize("geom", [(6, 4, 1, (1.0, 1.0)), (7, 7, 5, (0.5, 1.5))])
def test_apply_matches_oracle(sb, op, prec, tol, geom):
    n, p, seed, rr = geom
    w = wl.small_suspension(n, p, seed, radius_range=rr)
    g = ops.Geometry(w["centres"], w["radii"], p)
    dens = np.random.default_rng(seed + 30).normal(size=(g.N, 3))
    ref = ops.apply(g, op, dens)
    with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec) as s:
        out = s.apply(op, dens)
    assert np.all(_per_sphere(out, ref, g.npn) < tol)


@pytest.mark.parametrize("prec,tolF", [(0, 1e-8), (2, 1e-8), (1, 1e-6)])
def test_porous_solve_matches_oracle(sb, prec, tolF):
    w = wl.small_suspension(8, 6, 3, radius_range=(0.7, 1.3))
    g = ops.Geometry(w["centres"], w["radii"], 6)
    rng = np.random.default_rng(4)
    u0 = rng.normal(size=3)
    G = rng.normal(size=(3, 3))
    Fr, Tr, _ = osolve.solve_porous(g, u0, G, tol=1e-12)
    with sb.SphereBIE(w["centres"], w["radii"], 6, prec=prec, tol=1e-11) as s:
        F, T, info = s.porous(u0, G)
    assert info["status"] == 0 and info["rel_residual_true"] <= 1e-11
    for a, b in ((F, Fr), (T, Tr)):
        assert np.max(np.abs(a - b)) < tolF * np.max(np.abs(b))


def test_porous_single_sphere_drag(sb):
    a, U = 1.6, np.array([0.4, -1.0, 0.3])
    with sb.SphereBIE([[0.1, 0.2, 0.3]], [a], 6, prec=sb.SBIE_MIXED, tol=1e-12) as s:
        F, T, info = s.porous(U)
    np.testing.assert_allclose(F[0], -6 * math.pi * a * U, rtol=1e-9)
    assert np.max(np.abs(T)) < 1e-9


def _slip(x_nodes_normals, w, p):
    npn = (p + 1) * (2 * p + 2)
    ax = np.repeat(w["axes"], npn, axis=0)
    return wl.squirmer_slip(x_nodes_normals, ax, w["B1"], w["B2"])


@pytest.mark.parametrize("prec,tolv", [(0, 1e-8), (2, 1e-8), (1, 1e-6)])
def test_squirmer_solve_matches_oracle(sb, prec, tolv):
    p = 6
    w = wl.squirmers(6, p, seed=14, beta=-3.0, radius_range=(0.8, 1.2))
    g = ops.Geometry(w["centres"], w["radii"], p)
    slip = _slip(g.nrm, w, p)
    vr, wr, info_r = osolve.solve_squirmer(g, slip, tol=1e-12)
    with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec, tol=1e-11) as s:
        x, nrm, _ = s.nodes()
        np.testing.assert_allclose(nrm, g.nrm, atol=1e-14)
        v, om, info = s.squirmer(slip)
        dens = s.density()
    assert info["status"] == 0 and info["rel_residual_true"] <= 1e-11
    scale = max(np.max(np.abs(vr)), np.max(np.abs(wr)))
    assert np.max(np.abs(v - vr)) < tolv * scale and np.max(np.abs(om - wr)) < tolv * scale
    # the returned density is force- and torque-free on every sphere (Eq. 5.15)
    M0, M1 = ops.moments(g, dens)
    assert np.max(np.abs(M0)) < 1e-9 and np.max(np.abs(M1)) < 1e-9


def test_single_squirmer_speed(sb):
    p, a, B1 = 8, 0.9, 1.3
    e = np.array([1.0, 2.0, -2.0]) / 3.0
    with sb.SphereBIE([[0.0, 0.5, -0.2]], [a], p, prec=sb.SBIE_MIXED, tol=1e-12) as s:
        x, nrm, _ = s.nodes()
        slip = wl.squirmer_slip(nrm, np.repeat(e[None], len(nrm), axis=0), B1, 4.0)
        v, om, info = s.squirmer(slip)
    np.testing.assert_allclose(v[0], 2.0 / 3.0 * B1 * e, atol=1e-9)
    assert np.max(np.abs(om)) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_squirmers_equal_separate_contexts(sb, prec):
    """Squirmer suspensions of different sizes and orders in one batched
    context give the velocities of separate contexts."""
    specs = [(3, 4, 31), (5, 6, 32), (2, 5, 33)]
    ws = [wl.squirmers(n, p, seed=sd, beta=2.0) for (n, p, sd) in specs]
    slips = [_slip(ops.Geometry(w["centres"], w["radii"], p).nrm, w, p) for w, (n, p, sd) in zip(ws, specs)]
    with sb.SphereBIE(batch=[(w["centres"], w["radii"], p) for w, (n, p, sd) in zip(ws, specs)], prec=prec,
                      tol=1e-11) as s:
        v, om, info = s.squirmer(np.concatenate(slips))
    assert info["status"] == 0
    off = 0
    for w, (n, p, sd), sl in zip(ws, specs, slips):
        with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec, tol=1e-11) as s1:
            v1, w1, _ = s1.squirmer(sl)
        scale = max(np.max(np.abs(v1)), np.max(np.abs(w1)))
        assert np.max(np.abs(v[off:off + n] - v1)) < 1e-8 * scale
        assert np.max(np.abs(om[off:off + n] - w1)) < 1e-8 * scale
        off += n
