"""Pins of the two-sphere low-mode blocks and of the reference network's
gradients (the learned pair preconditioner)."""
import numpy as np
import pytest

from oracle import pairblock as pb
from oracle import signatures

L = 4


def test_low_mode_count_and_roundtrip():
    modes = pb.low_modes(L)
    assert len(modes) == 3 * (L + 1) ** 2 - 2 == 73
    a = np.random.default_rng(0).normal(size=73)
    np.testing.assert_allclose(pb.coef_to_low(pb.low_to_coef(a, L, 6), L), a)


@pytest.mark.parametrize("op,sig", [("resistance", signatures.D_plus), ("mobility", signatures.K_minus)])
def test_self_block_is_exterior_operator_above_degree_one(op, sig):
    """For n >= 2 the completion (N of Eq. 5.19, L of Eq. 5.8) carries no
    moment, so the self block of 1/2 I + D + N is diagonal with the exterior
    eigenvalues D+, and that of 1/2 I + K + L with K- (Theorem 2)."""
    B = pb.two_sphere_blocks([[0, 0, 0], [50.0, 0, 0]], [1.0, 1.0], 5, L, op=op)
    B00 = B[0, 0]
    modes = pb.low_modes(L)
    for j, (t, n, m, part) in enumerate(modes):
        if n < 2:
            continue
        col = B00[:, j]
        assert abs(col[j] - sig(n)[t]) < 1e-11
        assert np.max(np.abs(np.delete(col, j))) < 1e-11


@pytest.mark.parametrize("op", ["resistance", "mobility"])
def test_aligned_block_conserves_m(op):
    """Rotations about the pair axis commute with the operator: no coupling
    between different orders m in the pair frame."""
    B = pb.aligned_block(2.3, 1.0, 1.0, 5, L, op=op)
    modes = pb.low_modes(L)
    scale = np.max(np.abs(B))
    for i, (ti, ni, mi, pi_) in enumerate(modes):
        for j, (tj, nj, mj, pj) in enumerate(modes):
            if mi != mj:
                assert abs(B[i, j]) < 1e-11 * scale


def test_far_pair_block_expansion_matches_quadrature():
    """Well separated: the close-pair expansion and the smooth quadrature give
    the same block."""
    c = [[0, 0, 0], [0.3, -0.2, 6.0]]
    errs = []
    for p in (6, 8):
        Bn = pb.two_sphere_blocks(c, [1.0, 0.8], p, L, eta=1e9)[1, 0]
        Bf = pb.two_sphere_blocks(c, [1.0, 0.8], p, L, eta=0.0)[1, 0]
        errs.append(np.max(np.abs(Bn - Bf)) / np.max(np.abs(Bn)))
    assert errs[1] < errs[0] / 100 and errs[1] < 2e-8


def test_network_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    sizes = [5, 7, 6, 5, 4]
    params = []
    for i in range(4):
        params += [rng.normal(size=(sizes[i], sizes[i + 1])) * 0.5, rng.normal(size=sizes[i + 1]) * 0.1]
    X = rng.normal(size=(3, 5))
    Y = rng.normal(size=(3, 4))
    loss, grads = pb.mlp_loss_grad(params, X, Y)
    h = 1e-6
    for k in range(8):
        P = params[k]
        idx = tuple(rng.integers(0, s) for s in P.shape)
        P[idx] += h
        lp, _ = pb.mlp_loss_grad(params, X, Y)
        P[idx] -= 2 * h
        lm, _ = pb.mlp_loss_grad(params, X, Y)
        P[idx] += h
        assert abs((lp - lm) / (2 * h) - grads[k][idx]) < 1e-7
