"""Learned pair preconditioner: exact pair-frame blocks against the oracle,
network gradients against the reference back-propagation, and preconditioned
solves (exact blocks and trained network) that return the unpreconditioned
answer in fewer GMRES iterations."""
import numpy as np
import pytest

from oracle import pairblock as opb
from paper_1707_06551_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def _bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32)
    # round to nearest even on the upper 16 bits
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


@pytest.mark.parametrize("d,a_s,a_t,op", [(2.1, 1.0, 1.0, "resistance"), (2.6, 1.0, 1.0, "resistance"),
                                          (2.05, 0.8, 1.2, "resistance"), (2.1, 1.0, 1.0, "mobility"),
                                          (2.05, 1.2, 0.8, "mobility")])
def test_pair_blocks_match_oracle(sb, d, a_s, a_t, op):
    got = sb.sphere_bie_pair_blocks([d], a_s, a_t, 6, op)[0]
    ref = opb.aligned_block(d, a_s, a_t, 6, 4, op)
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))


def test_network_gradients_match_reference(sb):
    n_par = sb.sphere_bie_pair_network_size()
    rng = np.random.default_rng(0)
    sizes = [5, 128, 128, 128, 73 * 73]
    flat = []
    params = []
    for i in range(4):
        W = _bf16(rng.normal(size=(sizes[i], sizes[i + 1])) / np.sqrt(sizes[i]))
        b = (rng.normal(size=sizes[i + 1]) * 0.1).astype(np.float32)
        flat += [W.ravel(), b]
        params += [W.astype(np.float64), b.astype(np.float64)]
    flat = np.concatenate(flat)
    assert flat.size == n_par
    X = rng.normal(size=(6, 5)).astype(np.float32)
    Y = rng.normal(size=(6, 73 * 73)).astype(np.float32)
    loss, g = sb.sphere_bie_pair_network_gradients(flat, X, Y)
    lref, gref = opb.mlp_loss_grad(params, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - lref) < 1e-5 * lref
    off = 0
    for k in range(8):
        sz = gref[k].size
        gk = g[off:off + sz]
        off += sz
        assert np.max(np.abs(gk - gref[k].ravel())) < 2e-4 * np.max(np.abs(gref[k])) + 1e-9, k


def _suspension():
    w = wl.small_suspension(16, 6, 11, push=0.5, gap_range=(0.05, 0.2))
    return w["centres"], w["radii"], 6


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_pair_preconditioner(sb, prec):
    c, a, p = _suspension()
    rng = np.random.default_rng(3)
    v = rng.normal(size=(len(a), 3))
    w = rng.normal(size=(len(a), 3))
    with sb.SphereBIE(c, a, p, prec=prec, tol=1e-10) as s:
        F0, T0, i0 = s.resistance(v, w)
    with sb.SphereBIE(c, a, p, prec=prec, tol=1e-10, precond=2) as s:
        F1, T1, i1 = s.resistance(v, w)
    assert i0["status"] == 0 and i1["status"] == 0
    assert np.max(np.abs(F1 - F0)) < 1e-7 * np.max(np.abs(F0))
    assert i1["iters"] < 0.75 * i0["iters"], (i0["iters"], i1["iters"])


def test_learned_pair_preconditioner(sb, tmp_path):
    path = tmp_path / "pairnet.bin"
    info = sb.sphere_bie_train_pair_network(path, n_samples=3000, p=6, epochs=200, seed=5)
    assert info["val_rel_err"] < 0.01, info
    c, a, p = _suspension()
    rng = np.random.default_rng(4)
    v = rng.normal(size=(len(a), 3))
    w = rng.normal(size=(len(a), 3))
    with sb.SphereBIE(c, a, p, tol=1e-10) as s:
        F0, T0, i0 = s.resistance(v, w)
    with sb.SphereBIE(c, a, p, tol=1e-10, precond=2) as s:
        F2, T2, i2 = s.resistance(v, w)
        pi2 = sb.sphere_bie_precond_info(s.ctx)
    with sb.SphereBIE(c, a, p, tol=1e-10, precond=1, weights=path) as s:
        F1, T1, i1 = s.resistance(v, w)
        pi1 = sb.sphere_bie_precond_info(s.ctx)
    assert i1["status"] == 0 and np.max(np.abs(F1 - F0)) < 1e-7 * np.max(np.abs(F0))
    # pairs beyond the trained gap range (0.01 .. 0.5) are left out, not extrapolated
    assert pi2["kind"] == 2 and pi1["kind"] == 1 and pi2["dropped"] == 0
    assert pi1["pairs"] + pi1["dropped"] == pi2["pairs"] and pi1["pairs"] > 0
    # the network's gain over the unpreconditioned method, and its distance from exact blocks
    assert i1["iters"] < 0.8 * i0["iters"], (i0["iters"], i1["iters"], i2["iters"])
    assert i1["iters"] <= i2["iters"] + 3, (i1["iters"], i2["iters"])


def test_exact_pair_preconditioner_mobility(sb):
    c, a, p = _suspension()
    rng = np.random.default_rng(6)
    F, T = rng.normal(size=(len(a), 3)), rng.normal(size=(len(a), 3))
    with sb.SphereBIE(c, a, p, prec=1, tol=1e-10) as s:
        v0, w0, i0 = s.mobility(F, T)
    with sb.SphereBIE(c, a, p, prec=1, tol=1e-10, precond=2) as s:
        v1, w1, i1 = s.mobility(F, T)
        pm = sb.sphere_bie_precond_info(s.ctx, "mobility")
        pr = sb.sphere_bie_precond_info(s.ctx, "resistance")
    assert i1["status"] == 0 and pm["kind"] == 2 and pm["pairs"] > 0 and pr["kind"] == 0
    assert np.max(np.abs(v1 - v0)) < 1e-7 * np.max(np.abs(v0))
    assert i1["iters"] < 0.75 * i0["iters"], (i0["iters"], i1["iters"])


def test_learned_mobility_network_and_fallback(sb, tmp_path):
    both = tmp_path / "both.bin"
    res_only = tmp_path / "res.bin"
    info = sb.sphere_bie_train_pair_network(both, n_samples=2000, p=6, epochs=200, seed=9,
                                            ops=("resistance", "mobility"))
    assert info["val_rel_err"] < 0.01, info
    sb.sphere_bie_train_pair_network(res_only, n_samples=600, p=6, epochs=50, seed=9)
    c, a, p = _suspension()
    rng = np.random.default_rng(8)
    F, T = rng.normal(size=(len(a), 3)), rng.normal(size=(len(a), 3))
    with sb.SphereBIE(c, a, p, tol=1e-10) as s:
        v0, w0, i0 = s.mobility(F, T)
    with sb.SphereBIE(c, a, p, tol=1e-10, precond=1, weights=both) as s:
        v1, w1, i1 = s.mobility(F, T)
        pm = sb.sphere_bie_precond_info(s.ctx, "mobility")
    with sb.SphereBIE(c, a, p, tol=1e-10, precond=1, weights=res_only) as s:
        v2, w2, i2 = s.mobility(F, T)
        pf = sb.sphere_bie_precond_info(s.ctx, "mobility")
    assert pm["kind"] == 1 and i1["status"] == 0 and i1["iters"] < 0.8 * i0["iters"], (i0["iters"], i1["iters"])
    assert np.max(np.abs(v1 - v0)) < 1e-7 * np.max(np.abs(v0))
    # no mobility network in the file: the mobility solve runs unpreconditioned
    assert pf["kind"] == 0 and i2["iters"] == i0["iters"] and np.max(np.abs(v2 - v0)) < 1e-9 * np.max(np.abs(v0))


def test_resistance_256_headline_configuration(sb, tmp_path):
    """The timed configuration at full size: 256 spheres, p = 10, mixed
    precision, learned pair preconditioner, graph-launched cycles.  Forces and
    torques agree with the FP64-accurate (double-float) solve to 1e-6, and the
    reported residual is the FP64 residual of the returned density."""
    w = wl.resistance_256()
    path = tmp_path / "pairnet.bin"
    sb.sphere_bie_train_pair_network(path, n_samples=1024, p=w["p"], gap_min=0.01, gap_max=2.0, epochs=100, seed=3)
    with sb.SphereBIE(w["centres"], w["radii"], w["p"], prec=sb.SBIE_MIXED, tol=w["tol"], precond=1,
                      weights=path) as s:
        F, T, info = s.resistance(w["vel"], w["omega"], w["u0"], w["G"])
        psi = s.density()
        x, _, _ = s.nodes()
        pi = sb.sphere_bie_precond_info(s.ctx)
    # pairs whose gap falls outside the sampled training range are left out
    assert info["status"] == 0 and info["graph_cycles"] > 0 and pi["kind"] == 1
    assert pi["pairs"] + pi["dropped"] == 559 and pi["pairs"] >= 550
    with sb.SphereBIE(w["centres"], w["radii"], w["p"], prec=sb.SBIE_FP64_DF, tol=w["tol"]) as s:
        F64, T64, i64 = s.resistance(w["vel"], w["omega"], w["u0"], w["G"])
        # b = v + omega x (x - c) - u_inf(x) with u_inf = u0 + G x (spheres held fixed)
        b = -(w["u0"][None, :] + x @ w["G"].T)
        r = b - s.apply("resistance", psi)
    assert i64["status"] == 0 and info["iters"] < i64["iters"]
    # per-result bound: the mixed solve at 1e-8 against the FP64-accurate solve
    # to 1e-11 (two solves at 1e-8 differ by both of their errors)
    with sb.SphereBIE(w["centres"], w["radii"], w["p"], prec=sb.SBIE_FP64_DF, tol=1e-11) as s:
        Fr, Tr, ir = s.resistance(w["vel"], w["omega"], w["u0"], w["G"])
    assert ir["status"] == 0
    assert np.max(np.abs(F - Fr)) < 1e-6 * np.max(np.abs(Fr))
    assert np.max(np.abs(T - Tr)) < 1e-6 * np.max(np.abs(Tr))
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= w["tol"] and abs(rel - info["rel_residual_true"]) <= 0.1 * w["tol"]
