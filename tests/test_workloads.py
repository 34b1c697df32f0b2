"""The seeded workload generators are deterministic and produce valid geometry."""
import math

import numpy as np
import pytest

from paper_1707_06551_gb300 import workloads as wl


def _min_gap(c, a):
    d = np.linalg.norm(c[:, None] - c[None], axis=-1) - a[:, None] - a[None]
    np.fill_diagonal(d, np.inf)
    return d.min()


def test_mobility_8():
    w = wl.mobility_8()
    assert w["centres"].shape == (8, 3) and w["p"] == 6
    d = np.linalg.norm(w["centres"][:, None] - w["centres"][None], axis=-1)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2.5
    assert np.all((w["centres"] >= 0) & (w["centres"] <= 12))
    np.testing.assert_array_equal(wl.mobility_8()["forces"], w["forces"])


def test_resistance_256():
    w = wl.resistance_256()
    c, a = w["centres"], w["radii"]
    assert c.shape == (256, 3) and w["p"] == 10
    assert _min_gap(c, a) >= 0.05 - 1e-12
    L = (256 * 4 / 3 * math.pi / 0.10) ** (1 / 3)
    assert np.all((c >= 0) & (c <= L))
    d = np.linalg.norm(c[:, None] - c[None], axis=-1) - 2
    np.fill_diagonal(d, np.inf)
    close = np.sum(d.min(1) <= 0.2 + 1e-12)
    assert close >= 0.15 * 256
    assert w["G"][0, 1] == 1.0 and np.count_nonzero(w["G"]) == 1


def test_resistance_256_close_pair_count():
    """The oracle's close-pair list (negation of Eq. 4.5 at eta = 1) for the timed
    workload: 1,118 directed pairs, i.e. the 559 pair systems the GPU path's
    pair preconditioner builds for it (test_resistance_256_headline_configuration)
    and the close_pairs the bench reports."""
    from oracle import operators as ops
    w = wl.resistance_256()
    assert ops.Geometry(w["centres"], w["radii"], w["p"]).n_near_pairs() == 1118


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_suspension(seed):
    w = wl.small_suspension(12, 4, seed)
    assert _min_gap(w["centres"], w["radii"]) >= 0.05 - 1e-12


@pytest.mark.parametrize("poly,counts", [(False, [8, 27, 125, 729, 4913]), (True, [15, 71, 429, 2969, 22065])])
def test_lattice_sphere_counts_are_the_papers(poly, counts):
    """Sec. 6 lists n_b = 8 ... 4913 (vertices) and 15 ... 22065 (with face and
    centre spheres) for the lattices of 1 to 16 units per side."""
    assert [len(wl.lattice(m, 4, poly)["radii"]) for m in (1, 2, 4, 8, 16)] == counts


@pytest.mark.parametrize("q", [1, 4])
def test_lattice_gaps(q):
    """Vertex spheres of radius 1 - 2^-q, 2 apart: minimum gap 2^(1-q); with
    the hole-sized face and centre spheres the minimum gap is 2^-q and no two
    spheres overlap."""
    for poly, gap in ((False, 2.0 ** (1 - q)), (True, 2.0 ** (-q))):
        w = wl.lattice(3, q, poly)
        c, a = w["centres"], w["radii"]
        d = np.linalg.norm(c[:, None] - c[None], axis=2) - a[:, None] - a[None]
        np.fill_diagonal(d, np.inf)
        assert abs(d.min() - gap) < 1e-12
        assert np.isclose(a.max(), 1 - 2.0 ** (-q))


def test_smooth_density_is_seeded_and_smooth():
    """The operator-apply density of the close-pair benchmark: reproducible,
    one rigid motion per sphere plus plane waves of wave number <= 1, so its
    variation across a unit sphere is bounded by the rigid part and |k|."""
    rng = np.random.default_rng(0)
    c = np.array([[0.0, 0, 0], [5.0, 0, 0]])
    d = rng.normal(size=(2, 50, 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    x = (c[:, None, :] + d).reshape(-1, 3)
    u1 = wl.smooth_density(x, c, 50, seed=3)
    u2 = wl.smooth_density(x, c, 50, seed=3)
    assert u1.shape == (100, 3) and np.array_equal(u1, u2)
    assert not np.allclose(u1, wl.smooth_density(x, c, 50, seed=4))
    # without plane waves it is a rigid motion on each sphere: (u(x) - u(c)) . (x - c) = 0
    r = wl.smooth_density(x, c, 50, seed=3, modes=0).reshape(2, 50, 3)
    ctr = wl.smooth_density(np.repeat(c, 50, axis=0), c, 50, seed=3, modes=0).reshape(2, 50, 3)
    np.testing.assert_allclose(np.sum((r - ctr) * d, axis=2), 0.0, atol=1e-12)
