"""Pin of the signature table (Theorem 2, Eq. 3.12) by direct high-order
quadrature of the kernels on single VSH modes with the target at the north
pole, where kernel x area element is bounded (r = 2 sin(theta/2)), so a plain
Gauss-Legendre (theta) x trapezoid (phi) rule converges spectrally.  Modes with
|m| >= 2 vanish at the pole; m = 0, 1 cover every (n, type)."""
import numpy as np
import pytest

from oracle import signatures, sph

NT, NP = 96, 64


def _pole_integrals(n, m):
    u, wu = np.polynomial.legendre.leggauss(NT)
    th = 0.5 * np.pi * (u + 1.0)
    wth = 0.5 * np.pi * wu
    ph = 2 * np.pi * np.arange(NP) / NP
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    ct, st, cp, sp = np.cos(TH), np.sin(TH), np.cos(PH), np.sin(PH)
    Y, V, W, X = sph.vsh_tables(n, ct, st, cp, sp)
    y = np.stack([st * cp, st * sp, ct], -1)
    dA = (wth[:, None] * st) * (2 * np.pi / NP)
    x0 = np.array([0.0, 0.0, 1.0])
    r = x0 - y
    rn = np.linalg.norm(r, axis=-1)
    out = {}
    for name, Z in (("V", V[n][m]), ("W", W[n][m]), ("X", X[n][m])):
        Zv = np.stack(Z, -1)
        rz = np.einsum("abi,abi->ab", r, Zv)
        # Stokeslet (Eq. 2.19)
        S = (Zv / rn[..., None] + r * (rz / rn ** 3)[..., None]) / (8 * np.pi)
        # double layer with source normal y, sign of Theorem 2 (jump D+ - D- = 1)
        ry = np.einsum("abi,abi->ab", r, y)
        D = 3.0 / (4 * np.pi) * r * (rz * ry / rn ** 5)[..., None]
        # traction of S with target normal e_z (Eq. 2.22)
        rx = r[..., 2]
        K = -3.0 / (4 * np.pi) * r * (rz * rx / rn ** 5)[..., None]
        out[name] = tuple(np.sum(dA[..., None] * F, axis=(0, 1)) for F in (S, D, K))
    Yp, Vp, Wp, Xp = sph.vsh_tables(n, np.array(1.0), np.array(0.0), np.array(1.0), np.array(0.0))
    zpole = {"V": np.array(Vp[n][m], complex), "W": np.array(Wp[n][m], complex), "X": np.array(Xp[n][m], complex)}
    return out, zpole


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("m", [0, 1])
def test_signatures_by_pole_quadrature(n, m):
    ints, z = _pole_integrals(n, m)
    lamS = signatures.S(n)
    lamD = signatures.D_pv(n)
    lamK = signatures.K_pv(n)
    for t, name in enumerate("VWX"):
        if np.max(np.abs(z[name])) < 1e-14:
            continue
        S, D, K = ints[name]
        np.testing.assert_allclose(S, lamS[t] * z[name], atol=1e-12)
        np.testing.assert_allclose(D, lamD[t] * z[name], atol=1e-12)
        np.testing.assert_allclose(K, lamK[t] * z[name], atol=1e-12)


def test_n0_single_layer_and_double_layer_of_radial_field():
    """V_0 = -Y_0 e_r: S[e_r] = 0 (incompressible radial flow), D PV on e_r = 1/2."""
    ints, z = _pole_integrals(0, 0)
    S, D, K = ints["V"]
    np.testing.assert_allclose(S, 0.0, atol=1e-13)
    np.testing.assert_allclose(D, signatures.D_pv(0)[0] * z["V"], atol=1e-12)
    assert abs(signatures.D_pv(0)[0] - 0.5) < 1e-15


@pytest.mark.parametrize("n", range(0, 9))
def test_jumps(n):
    dp, dm = signatures.D_plus(n), signatures.D_minus(n)
    kp, km = signatures.K_plus(n), signatures.K_minus(n)
    for t in range(3):
        if n == 0 and t > 0:
            continue
        assert abs(dp[t] - dm[t] - 1.0) < 1e-14
        assert abs(kp[t] - km[t] + 1.0) < 1e-14


def test_rigid_null_space_of_exterior_D_and_interior_K():
    """D+ (= 1/2 + D_pv) and K- (= 1/2 + K_pv) vanish on W_1 and X_1 (Eq. 5.8)."""
    assert abs(signatures.D_plus(1)[1]) < 1e-15 and abs(signatures.D_plus(1)[2]) < 1e-15
    assert abs(0.5 + signatures.K_pv(1)[1]) < 1e-15 and abs(0.5 + signatures.K_pv(1)[2]) < 1e-15
