"""Pins of the oracle's rotated-frame close-pair scheme (Sec. 4.2, Fig. 2):
its frame, and agreement with the direct evaluation of the exterior formulas
(oracle.operators.near_term, itself pinned) -- to rounding when the field on
the target sphere is resolved at degree p, and converging spectrally in p
for close pairs, where stage (3) projects onto degree <= p."""
import numpy as np
import pytest

from oracle import fftnear, offsurface, operators as ops, vsh


def _density(p, seed):
    c = np.zeros((3, p + 1, p + 1), complex)
    rng = np.random.default_rng(seed)
    for t in range(3):
        for n in range(p + 1):
            if t > 0 and n == 0:
                continue
            # algebraic decay, as the paper's synthetic data (Sec. 6)
            c[t, n, 0] = rng.normal() / (1 + n) ** 2
            c[t, n, 1:n + 1] = (rng.normal(size=n) + 1j * rng.normal(size=n)) / (1 + n) ** 2
    return c


def _direct(op, c, a_s, c_s, c_t, a_t, p):
    ct, st, cp, sp = vsh.grid_angles(p)
    dirs = np.stack([st * cp, st * sp, ct], axis=-1).reshape(-1, 3)
    x = np.asarray(c_t)[None, :] + a_t * dirs
    xh = (x - np.asarray(c_s)[None, :]) / a_s
    if op == "S":
        return a_s * offsurface.S_velocity(c, xh)
    if op == "D":
        return offsurface.D_velocity(c, xh)
    return offsurface.S_traction(c, xh, dirs)


@pytest.mark.parametrize("v", [[1.0, 2.0, -0.5], [0.0, 0.0, 3.0], [0.0, 0.0, -2.0], [-1.0, 0.0, 0.0]])
def test_pair_frame(v):
    Q, d = fftnear.pair_frame(np.zeros(3), v)
    np.testing.assert_allclose(Q @ Q.T, np.eye(3), atol=1e-15)
    np.testing.assert_allclose(np.linalg.det(Q), 1.0, atol=1e-15)
    np.testing.assert_allclose(Q @ np.asarray(v), [0.0, 0.0, d], atol=1e-14)


@pytest.mark.parametrize("op", ["S", "D", "K"])
def test_resolved_field_matches_direct(op):
    """A source 10 radii away: the field on the target sphere is resolved at
    p = 12 (its degree-n content falls like (a_t / d)^n), so projecting it
    onto degree <= 12 changes nothing at the 1e-9 level."""
    p = 12
    c = _density(p, 1)
    cs, ct_ = np.array([0.1, -0.2, 0.3]), np.array([0.1, -0.2, 0.3]) + 10.0 * np.array([0.48, 0.6, 0.64])
    got = fftnear.near_pair(op, c, 1.0, cs, ct_, 1.0, p)
    ref = _direct(op, c, 1.0, cs, ct_, 1.0, p)
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("op", ["S", "D", "K"])
def test_close_pair_converges_to_direct(op):
    """Gap 0.3 between radii 1.0 and 0.8: the difference to the direct
    evaluation falls geometrically with p (by at least 10 per 6 orders)."""
    cs, ct_ = np.zeros(3), np.array([1.2, -0.9, 1.0])
    ct_ = ct_ / np.linalg.norm(ct_) * 2.1
    errs = []
    for p in (6, 12, 20):
        c = _density(p, 2)
        c[:, 7:, :] = 0.0  # the same density at every p
        got = fftnear.near_pair(op, c, 1.0, cs, ct_, 0.8, p)
        ref = _direct(op, c, 1.0, cs, ct_, 0.8, p)
        errs.append(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert errs[2] < 1e-4 and errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


def test_operator_converges_to_direct_on_a_suspension():
    """Three spheres, every pair close (gaps 1.1 to 1.4 radii), a random nodal
    density: the rotated-scheme resistance, mobility, porous-media and
    squirmer operators approach the direct ones (oracle.operators.apply)
    geometrically in p."""
    c = np.array([[0.0, 0.0, 0.0], [3.2, 0.4, -0.3], [-0.5, 3.3, 0.2]])
    errs = {"resistance": [], "mobility": [], "porous": [], "squirmer": []}
    for p in (8, 12, 16):
        g = ops.Geometry(c, [1.0, 0.9, 1.1], p, eta=2.0)
        assert g.n_near_pairs() == 6
        dens = np.random.default_rng(4).normal(size=(g.N, 3))
        for op in errs:
            got = fftnear.apply(g, op, dens)
            ref = ops.apply(g, op, dens)
            errs[op].append(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    for op, e in errs.items():
        assert e[2] < 1e-5 and e[1] < e[0] / 10 and e[2] < e[1] / 10, (op, e)
