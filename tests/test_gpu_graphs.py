"""Device-resident GMRES restart cycles: a cycle run as one CUDA graph launch
(WHILE node over the Arnoldi iteration) gives the iterates of the same cycle
stepped from the host, for single problems, batches of uneven problems,
mixed precision and the pair preconditioner; stopping at max_iter and
reuse of a captured cycle across solves and retuning behave as without
graphs."""
import numpy as np
import pytest

from oracle import solve as osolve
from oracle import operators as ops
from paper_1707_06551_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def _err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _geom(n=9, p=6, seed=5):
    w = wl.small_suspension(n, p, seed, radius_range=(0.5, 1.5))
    return w["centres"], w["radii"], p


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_graph_cycle_equals_host_stepped(sb, prec):
    c, a, p = _geom()
    rng = np.random.default_rng(21)
    v, w = rng.normal(size=(len(a), 3)), rng.normal(size=(len(a), 3))
    out = {}
    for graphs in (False, True):
        with sb.SphereBIE(c, a, p, prec=prec, tol=1e-10, restart=8, graphs=graphs) as s:
            out[graphs] = s.resistance(v, w)
    (F0, T0, i0), (F1, T1, i1) = out[False], out[True]
    assert i0["graph_cycles"] == 0 and i1["graph_cycles"] == i1["restarts"] > 1
    assert i1["status"] == 0 and abs(i1["iters"] - i0["iters"]) <= 1
    assert _err(F1, F0) < 1e-8 and _err(T1, T0) < 1e-8


def test_graph_solve_matches_oracle(sb):
    w8 = wl.mobility_8()
    g = ops.Geometry(w8["centres"], w8["radii"], w8["p"])
    vr, wr, _ = osolve.solve_mobility(g, w8["forces"], w8["torques"], tol=1e-12)
    with sb.SphereBIE(w8["centres"], w8["radii"], w8["p"], tol=1e-11) as s:
        v, w, info = s.mobility(w8["forces"], w8["torques"])
        v2, w2, info2 = s.mobility(w8["forces"], w8["torques"])  # the captured cycle is reused
    assert info["status"] == 0 and info["graph_cycles"] >= 1
    assert _err(v, vr) < 1e-8 and _err(w, wr) < 1e-8
    assert info2["iters"] == info["iters"] and np.array_equal(v2, v)


def test_graph_batch_of_uneven_problems(sb):
    batch = []
    for n, p, seed in [(3, 4, 1), (5, 6, 2), (1, 3, 3), (6, 5, 5)]:
        w = wl.small_suspension(n, p, seed, radius_range=(0.7, 1.3))
        batch.append((w["centres"], w["radii"], p))
    rng = np.random.default_rng(8)
    F = rng.normal(size=(sum(len(b[1]) for b in batch), 3))
    T = rng.normal(size=F.shape)
    res = {}
    for graphs in (False, True):
        with sb.SphereBIE(batch=batch, prec=1, tol=1e-10, graphs=graphs) as s:
            res[graphs] = s.mobility(F, T)
    (v0, w0, i0), (v1, w1, i1) = res[False], res[True]
    assert i1["graph_cycles"] > 0 and i1["status"] == 0 and i1["rel_residual_true"] <= 1e-10
    assert _err(v1, v0) < 1e-7 and _err(w1, w0) < 1e-7


def test_graph_with_pair_preconditioner(sb):
    w = wl.small_suspension(12, 6, 11, push=0.5, gap_range=(0.05, 0.2))
    c, a = w["centres"], w["radii"]
    rng = np.random.default_rng(3)
    v, om = rng.normal(size=(len(a), 3)), rng.normal(size=(len(a), 3))
    res = {}
    for graphs in (False, True):
        with sb.SphereBIE(c, a, 6, tol=1e-10, precond=2, graphs=graphs) as s:
            res[graphs] = s.resistance(v, om)
    (F0, _, i0), (F1, _, i1) = res[False], res[True]
    assert i1["graph_cycles"] > 0 and i1["status"] == 0 and abs(i1["iters"] - i0["iters"]) <= 1
    assert _err(F1, F0) < 1e-8


def test_graph_stops_at_max_iter(sb):
    c, a, p = _geom(6, 4, 1)
    with sb.SphereBIE(c, a, p, tol=1e-14, max_iter=5, restart=3) as s:
        F, T, info = s.resistance(np.ones((len(a), 3)), np.zeros((len(a), 3)))
    assert info["status"] == sb.SBIE_ERR_NOT_CONVERGED and info["iters"] == 5
    assert info["graph_cycles"] == 2 and np.all(np.isfinite(F))


def test_graph_recaptured_after_autotune(sb):
    c, a, p = _geom(7, 9, 7)
    rng = np.random.default_rng(5)
    v, w = rng.normal(size=(len(a), 3)), rng.normal(size=(len(a), 3))
    with sb.SphereBIE(c, a, p, prec=1, tol=1e-10) as s:
        F0, _, i0 = s.resistance(v, w)
        sb.sphere_bie_autotune(s.ctx, "resistance")
        F1, _, i1 = s.resistance(v, w)
    assert i0["graph_cycles"] > 0 and i1["graph_cycles"] > 0
    assert i1["status"] == 0 and _err(F1, F0) < 1e-8
