"""The rotated, FFT-accelerated close-pair scheme (Sec. 4.2, Fig. 2; opts
near_scheme = 1) on the CUDA path against the oracle's restatement of its
three stages (oracle.fftnear): operator applies per sphere to 1e-10 on small
suspensions with close pairs, and on sampled spheres of the dense suspension
(1,024 spheres, 13,940 close pairs) at p = 12 and 16, in FP64 (1e-10) and in
the FP32 operator of the mixed path (2e-5); solves with it converge to the
solves of the direct scheme as p grows, in FP64 and in mixed precision."""
import numpy as np
import pytest

from oracle import fftnear
from oracle import operators as ops
from paper_1707_06551_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


def _per_sphere(got, ref, npn):
    return np.max(np.abs(got - ref).reshape(-1, npn, 3), axis=(1, 2)) / np.max(
        np.abs(ref).reshape(-1, npn, 3), axis=(1, 2))


@pytest.mark.parametrize("op", ["S", "D", "K", "resistance", "mobility", "porous", "squirmer"])
@pytest.mark.parametrize("geom", [(6, 4, 1, (1.0, 1.0)), (7, 9, 5, (0.5, 1.5))])
def test_rotated_scheme_matches_oracle(sb, op, geom):
    n, p, seed, rr = geom
    w = wl.small_suspension(n, p, seed, radius_range=rr)
    g = ops.Geometry(w["centres"], w["radii"], p)
    assert g.n_near_pairs() > 0
    dens = np.random.default_rng(seed + 60).normal(size=(g.N, 3))
    ref = fftnear.apply(g, op, dens)
    for prec, tol in ((0, 1e-10), (1, 2e-5)):
        with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec, near_scheme=1) as s:
            out = s.apply(op, dens)
        assert np.all(_per_sphere(out, ref, g.npn) < tol), (prec, _per_sphere(out, ref, g.npn).max())


@pytest.mark.parametrize("p,prec,tol", [(12, 0, 1e-10), (16, 0, 1e-10), (12, 1, 2e-5), (16, 1, 2e-5)])
def test_dense_1024_rotated_scheme_sampled(sb, p, prec, tol):
    """The mobility operator (Eq. 5.8) of the dense suspension with the rotated
    close-pair scheme, on its sphere with the most close partners: FP64, and
    the FP32 operator of the mixed path (FP32 rotated scheme and far field)."""
    w = wl.dense_1024()
    g = ops.Geometry(w["centres"], w["radii"], p)
    nc = [len(x) for x in g.near]
    sample = [int(np.argmax(nc))]
    rows = np.concatenate([np.arange(g.sl(i).start, g.sl(i).stop) for i in sample])
    dens = np.random.default_rng(p).normal(size=(g.N, 3))
    ref = fftnear.apply(g, "mobility", dens, sample)[rows]
    with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec, near_scheme=1) as s:
        out = s.apply("mobility", dens)[rows]
    assert np.all(_per_sphere(out, ref, g.npn) < tol), _per_sphere(out, ref, g.npn).max()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-8)])
def test_rotated_scheme_solves_converge_to_direct(sb, prec, tol):
    """Resistance solves of a suspension with gaps 0.05-0.3: the forces with the
    rotated scheme approach those of the direct scheme as p grows (the
    scheme's projection error falls spectrally), in FP64 and in mixed
    precision (the FP32 operator with the FP32 rotated scheme inside
    iterative refinement on the FP64-accurate operator with the FP64 one)."""
    w = wl.small_suspension(6, 4, 3)
    v = np.random.default_rng(2).normal(size=(6, 3))
    errs = []
    for p in (6, 10, 14):
        F = {}
        for scheme in (0, 1):
            with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec, tol=tol, near_scheme=scheme) as s:
                F[scheme], _, info = s.resistance(v, np.zeros((6, 3)))
                assert info["status"] == 0
        errs.append(np.max(np.abs(F[1] - F[0])) / np.max(np.abs(F[0])))
    assert errs[2] < errs[0] / 10 and errs[2] < 1e-3, errs


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_batch_with_rotated_scheme_equals_separate_contexts(sb, prec, tol):
    """A batch of suspensions of different orders with the rotated scheme
    applies each problem's operator as a context of its own does."""
    batch = []
    for n, p, seed in ((4, 4, 1), (5, 6, 2), (3, 5, 3)):
        w = wl.small_suspension(n, p, seed, radius_range=(0.8, 1.2))
        batch.append((w["centres"], w["radii"], p))
    rng = np.random.default_rng(11)
    dens = [rng.normal(size=(len(r) * (p + 1) * (2 * p + 2), 3)) for (c, r, p) in batch]
    with sb.SphereBIE(batch=batch, prec=prec, near_scheme=1) as s:
        out = s.apply("mobility", np.concatenate(dens))
    off = 0
    for (c, r, p), d in zip(batch, dens):
        with sb.SphereBIE(c, r, p, prec=prec, near_scheme=1) as s1:
            ref = s1.apply("mobility", d)
        got = out[off:off + len(d)]
        off += len(d)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("op", ["S", "D", "K", "mobility"])
def test_rotated_scheme_at_p24(sb, op):
    """The library's largest order: the evaluation kernel reads the pair's
    channels from global memory and needs 210 KB of shared memory in FP64."""
    w = wl.small_suspension(3, 24, 5, radius_range=(0.8, 1.2))
    g = ops.Geometry(w["centres"], w["radii"], 24)
    assert g.n_near_pairs() > 0
    dens = np.random.default_rng(24).normal(size=(g.N, 3))
    ref = fftnear.apply(g, op, dens)
    for prec, tol in ((0, 1e-10), (1, 2e-5)):
        with sb.SphereBIE(w["centres"], w["radii"], 24, prec=prec, near_scheme=1) as s:
            out = s.apply(op, dens)
        assert np.all(_per_sphere(out, ref, g.npn) < tol), (prec, _per_sphere(out, ref, g.npn).max())
