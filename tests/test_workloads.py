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
