"""The lattices of the operator-apply scaling tests (Sec. 6): the double layer
and the traction of the single layer on the CUDA path against the oracle on
sampled target spheres of a densely packed polydisperse lattice (q = 4, gaps
down to 1/16, a vertex, a face and a centre sphere sampled) and of a loosely
packed monodisperse one (q = 1).  Per-sphere bounds as in the other parity
tests: FP64 and double-float 1e-10, mixed precision 2e-5."""
import numpy as np
import pytest

from oracle import operators as ops
from paper_1707_06551_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    from paper_1707_06551_gb300 import build_lib
    build_lib.build()
    from paper_1707_06551_gb300 import sphere_bie
    return sphere_bie


@pytest.mark.parametrize("m,q,poly,p", [(2, 4, True, 4), (4, 1, False, 8)])
@pytest.mark.parametrize("op", ["D", "K"])
def test_lattice_sampled_parity(sb, m, q, poly, p, op):
    w = wl.lattice(m, q, poly)
    g = ops.Geometry(w["centres"], w["radii"], p)
    a = g.a
    sample = [0, int(np.argmin(a)), int(np.argmax(np.arange(g.n) * (a < a.max())))] if poly else [0, g.n // 2]
    sample = sorted(set(sample))
    rows = np.concatenate([np.arange(g.sl(i).start, g.sl(i).stop) for i in sample])
    dens = np.random.default_rng(m + q).normal(size=(g.N, 3))
    ref = ops.apply_at(g, op, dens, sample)[rows].reshape(-1, g.npn, 3)
    for prec, tol in ((0, 1e-10), (2, 1e-10), (1, 2e-5)):
        with sb.SphereBIE(w["centres"], w["radii"], p, prec=prec) as s:
            out = s.apply(op, dens)[rows].reshape(-1, g.npn, 3)
        err = np.max(np.abs(out - ref), axis=(1, 2)) / np.max(np.abs(ref), axis=(1, 2))
        assert np.all(err < tol), (prec, err)
