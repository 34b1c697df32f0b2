"""The Laplace family and the magnetostatic problem (Problem 3) on the CUDA
path against the oracle: the single layer, double layer and flux operators on
suspensions with close pairs (1e-10 per sphere, FP64), the coupled
magnetic + mobility solve (forces, torques and rigid motions), and the closed
forms the oracle is pinned to."""
import numpy as np
import pytest

from oracle import laplace as olap
from oracle import operators as ops
from oracle import solve as osolve
from paper_1707_06551_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


GEOMS = [(6, 4, 1, (1.0, 1.0)), (7, 7, 5, (0.5, 1.5)), (3, 1, 2, (1.0, 1.0))]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("op", ["SL", "DL", "KL"])
@pytest.mark.parametrize("geom", GEOMS)
def test_laplace_layers_match_oracle(sb, op, geom, prec):
    n, p, seed, rr = geom
    w = wl.small_suspension(n, p, seed, radius_range=rr)
    g = ops.Geometry(w["centres"], w["radii"], p)
    q = np.random.default_rng(seed + 50).normal(size=g.N)
    ref = olap.layer(g, op, q)
    with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec) as s:
        out = s.laplace(op, q)
    got, exp = out.reshape(-1, g.npn), ref.reshape(-1, g.npn)
    err = np.max(np.abs(got - exp), axis=1) / np.max(np.abs(exp), axis=1)
    assert np.all(err < 1e-10), err


@pytest.mark.parametrize("prec,tol", [(0, 1e-8), (1, 1e-6)])
def test_mhd_solve_matches_oracle(sb, prec, tol):
    w = wl.small_suspension(5, 6, 7, radius_range=(0.8, 1.2))
    g = ops.Geometry(w["centres"], w["radii"], 6)
    H0, eta = np.array([0.4, -0.2, 1.1]), 0.6
    Fr, Tr, vr, wr, _ = osolve.solve_mhd(g, H0, eta, tol=1e-12)
    with sb.SphereBIE(w["centres"], w["radii"], 6, prec=prec, tol=1e-12) as s:
        F, T, v, om, info = s.mhd(H0, eta)
    assert info["status"] == 0 and info["rel_residual_true"] <= 1e-12
    for a, b in ((F, Fr), (T, Tr), (v, vr), (om, wr)):
        assert np.max(np.abs(a - b)) < tol * np.max(np.abs(b)), (np.max(np.abs(a - b)), np.max(np.abs(b)))


def test_single_permeable_sphere_feels_no_force(sb):
    with sb.SphereBIE([[0.1, 0.2, 0.3]], [1.3], 6, tol=1e-12) as s:
        F, T, v, om, info = s.mhd([0.0, 0.5, 1.0], 0.8)
    assert np.max(np.abs(F)) < 1e-10 and np.max(np.abs(T)) < 1e-10
    assert np.max(np.abs(v)) < 1e-10 and np.max(np.abs(om)) < 1e-10


def test_two_spheres_along_the_field_attract(sb):
    with sb.SphereBIE([[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]], [1.0, 1.0], 8, tol=1e-12) as s:
        F, T, v, om, info = s.mhd([0.0, 0.0, 2.0], 0.7)
    assert F[0][2] > 0 > F[1][2] and v[0][2] > 0 > v[1][2]
    np.testing.assert_allclose(F[0], -F[1], atol=1e-10 * abs(F[0][2]))
