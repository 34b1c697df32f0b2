"""Batched contexts (many independent suspensions of uneven size and VSH
order in one context): operator applies and solves equal those of separate
single-problem contexts, and match the oracle problem by problem."""
import numpy as np
import pytest

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


def _batch():
    specs = [(3, 4, 1), (5, 6, 2), (1, 3, 3), (4, 4, 4), (6, 5, 5), (2, 6, 6)]  # (n, p, seed)
    out = []
    for n, p, seed in specs:
        w = wl.small_suspension(n, p, seed, radius_range=(0.7, 1.3))
        out.append((w["centres"], w["radii"], p))
    return out


def _err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("op", ["K", "resistance", "mobility"])
def test_batch_apply_equals_separate_contexts(sb, op, prec):
    batch = _batch()
    rng = np.random.default_rng(7)
    dens = [rng.normal(size=(len(r) * (p + 1) * (2 * p + 2), 3)) for (c, r, p) in batch]
    with sb.SphereBIE(batch=batch, prec=prec) as s:
        assert s.N == sum(len(d) for d in dens)
        out = s.apply(op, np.concatenate(dens))
    off = 0
    for (c, r, p), d in zip(batch, dens):
        with sb.SphereBIE(c, r, p, prec=prec) as s1:
            ref = s1.apply(op, d)
        got = out[off:off + len(d)]
        off += len(d)
        assert _err(got, ref) < (1e-12 if prec != 1 else 1e-6)


def test_batch_apply_matches_oracle(sb):
    batch = _batch()
    rng = np.random.default_rng(8)
    dens = [rng.normal(size=(len(r) * (p + 1) * (2 * p + 2), 3)) for (c, r, p) in batch]
    with sb.SphereBIE(batch=batch) as s:
        out = s.apply("resistance", np.concatenate(dens))
        x, nrm, w = s.nodes()
    off = 0
    for (c, r, p), d in zip(batch, dens):
        g = ops.Geometry(c, r, p)
        ref = ops.apply(g, "resistance", d)
        assert _err(out[off:off + len(d)], ref) < 1e-10
        np.testing.assert_allclose(x[off:off + len(d)], g.x, atol=1e-13)
        np.testing.assert_allclose(w[off:off + len(d)], g.w, atol=1e-13)
        off += len(d)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_solves_match_per_problem_oracle(sb, prec):
    batch = _batch()
    rng = np.random.default_rng(9)
    F = [rng.normal(size=(len(r), 3)) for (c, r, p) in batch]
    T = [rng.normal(size=(len(r), 3)) for (c, r, p) in batch]
    with sb.SphereBIE(batch=batch, prec=prec, tol=1e-11) as s:
        v, w, info = s.mobility(np.concatenate(F), np.concatenate(T))
        assert info["status"] == 0 and info["rel_residual_true"] <= 1e-11
        Fr, Tr, info2 = s.resistance(v, w)
        assert info2["status"] == 0
    off = 0
    for (c, r, p), f, t in zip(batch, F, T):
        g = ops.Geometry(c, r, p)
        vr, wr, _ = osolve.solve_mobility(g, f, t, tol=1e-12)
        k = len(r)
        tolv = 1e-8 if prec != 1 else 1e-6
        assert _err(v[off:off + k], vr) < tolv and _err(w[off:off + k], wr) < tolv
        Fo, To, _ = osolve.solve_resistance(g, v[off:off + k], w[off:off + k], tol=1e-12)
        assert _err(Fr[off:off + k], Fo) < tolv and _err(Tr[off:off + k], To) < tolv
        off += k
