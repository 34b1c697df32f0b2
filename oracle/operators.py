"""Discrete boundary integral operators for N rigid spheres (Sec. 4.1, 4.3;
Problems 2 and 5 of Sec. 5).  Test infrastructure only.

An operator apply splits into (Sec. 4.3):
  self  analysis -> signature (Theorem 2) -> synthesis on the same sphere (Sec. 4.1, Eqs. 4.6-4.7);
  far   the smooth quadrature (Eq. 4.4) over nodes of every well-separated sphere (Eq. 4.5);
  near  the exterior expansion of each close source sphere evaluated at the
        target nodes (Sec. 4.1, Eqs. 3.6-3.11, 3.18).

Readings of points the paper leaves open (each also listed in the design notes):
  * close pairs: sphere k is near sphere i (i != k) when
      |c_i - c_k| - a_i - a_k < eta * max(2 a_i, 2 a_k)       (negation of Eq. 4.5);
  * radius scaling: the signatures and exterior formulas are for the unit
    sphere; S scales by the source radius a, D and K are scale free;
  * the self term of D and K is the principal value (D+ + D-)/2, and the 1/2 I
    of the BIEs is added nodally;
  * L_k (Eq. 5.8) acts on Gamma_k only, about the centre of sphere k;
  * N_k (Eq. 5.19) is a Stokeslet of strength int psi and a rotlet of strength
    int (y - c_k) x psi, both at c_k, evaluated at every node.
"""
import numpy as np

from . import kernels, offsurface, quadrature, signatures, vsh


class OverlapError(ValueError):
    pass


class Geometry:
    def __init__(self, centres, radii, p, eta=1.0):
        self.c = np.asarray(centres, float).reshape(-1, 3)
        self.a = np.asarray(radii, float).reshape(-1)
        self.p = int(p)
        self.eta = float(eta)
        n = len(self.a)
        self.n = n
        if p < 1:
            raise ValueError("p >= 1 required")
        if np.any(self.a <= 0):
            raise ValueError("radii must be positive")
        self.npn = (p + 1) * (2 * p + 2)
        xs, ns, ws = [], [], []
        for i in range(n):
            x, nr, w = quadrature.sphere_nodes(self.c[i], self.a[i], p)
            xs.append(x)
            ns.append(nr)
            ws.append(w)
        self.x = np.concatenate(xs)
        self.nrm = np.concatenate(ns)
        self.w = np.concatenate(ws)
        # one row of gaps |c_i - c_k| - a_i - a_k per target sphere i
        self.near = [[] for _ in range(n)]
        for i in range(n):
            gap = np.sqrt(np.sum((self.c[i][None, :] - self.c) ** 2, axis=1)) - self.a[i] - self.a
            gap[i] = np.inf
            bad = np.nonzero(gap <= 0)[0]
            if len(bad):
                raise OverlapError(f"spheres {i} and {int(bad[0])} overlap or touch")
            self.near[i] = [int(k) for k in np.nonzero(gap < self.eta * 2.0 * np.maximum(self.a[i], self.a))[0]]

    @property
    def N(self):
        return self.n * self.npn

    def sl(self, i):
        return slice(i * self.npn, (i + 1) * self.npn)

    def n_near_pairs(self):
        return sum(len(v) for v in self.near)


def _signature(op, n, a):
    if op == "S":
        s = signatures.S(n)
        return tuple(a * v for v in s)
    if op == "D":
        return signatures.D_pv(n)
    if op == "K":
        return signatures.K_pv(n)
    raise ValueError(op)


def coefficients(g, dens):
    """VSH coefficients of the density on every sphere (as a function on the unit sphere)."""
    return [vsh.analysis(dens[g.sl(i)], g.p) for i in range(g.n)]


def _targets(g, targets):
    return range(g.n) if targets is None else list(targets)


def self_term(g, op, dens, coefs=None, targets=None):
    """Self interaction: synthesis of (signature x coefficients), Sec. 4.1 (Eqs. 4.6-4.7)."""
    coefs = coefficients(g, dens) if coefs is None else coefs
    out = np.zeros_like(dens)
    for i in _targets(g, targets):
        c = coefs[i].copy()
        for n in range(g.p + 1):
            lam = _signature(op, n, g.a[i])
            for t in range(3):
                c[t, n, :] *= lam[t]
        c[1, 0, 0] = 0.0
        c[2, 0, 0] = 0.0
        out[g.sl(i)] = vsh.synthesis(c)
    return out


def far_term(g, op, dens, targets=None):
    """Smooth quadrature (Eq. 4.4) over all nodes of well-separated spheres."""
    out = np.zeros_like(dens)
    dw = dens * g.w[:, None]
    for i in _targets(g, targets):
        excl = set(g.near[i]) | {i}
        src = np.concatenate([np.arange(g.sl(k).start, g.sl(k).stop) for k in range(g.n) if k not in excl]
                             ) if len(excl) < g.n else np.zeros(0, int)
        if len(src) == 0:
            continue
        xt = g.x[g.sl(i)]
        if op == "S":
            out[g.sl(i)] = kernels.stokeslet_sum(xt, g.x[src], dw[src])
        elif op == "D":
            out[g.sl(i)] = kernels.stresslet_sum_D(xt, g.x[src], g.nrm[src], dw[src])
        elif op == "K":
            out[g.sl(i)] = kernels.stresslet_sum_K(xt, g.nrm[g.sl(i)], g.x[src], dw[src])
        else:
            raise ValueError(op)
    return out


def near_term(g, op, dens, coefs=None, targets=None):
    """Exterior expansion of each close source sphere at the target nodes (Sec. 4.1)."""
    coefs = coefficients(g, dens) if coefs is None else coefs
    out = np.zeros_like(dens)
    for i in _targets(g, targets):
        xt = g.x[g.sl(i)]
        for k in g.near[i]:
            xh = (xt - g.c[k][None, :]) / g.a[k]
            if op == "S":
                out[g.sl(i)] += g.a[k] * offsurface.S_velocity(coefs[k], xh)
            elif op == "D":
                out[g.sl(i)] += offsurface.D_velocity(coefs[k], xh)
            elif op == "K":
                out[g.sl(i)] += offsurface.S_traction(coefs[k], xh, g.nrm[g.sl(i)])
            else:
                raise ValueError(op)
    return out


def layer(g, op, dens, targets=None):
    """Raw sum over k of S_k, D_k or K_k at every node (self by its signature);
    with `targets`, only the rows of those target spheres are filled."""
    dens = np.asarray(dens, float).reshape(-1, 3)
    if targets is None:
        coefs = coefficients(g, dens)
    else:
        need = set(targets)
        for i in targets:
            need |= set(g.near[i])
        coefs = [vsh.analysis(dens[g.sl(k)], g.p) if k in need else None for k in range(g.n)]
    return (self_term(g, op, dens, coefs, targets) + far_term(g, op, dens, targets)
            + near_term(g, op, dens, coefs, targets))


def moments(g, dens):
    """Per sphere M0 = int psi and M1 = int (y - c_k) x psi by the node quadrature."""
    dens = np.asarray(dens, float).reshape(-1, 3)
    M0 = np.zeros((g.n, 3))
    M1 = np.zeros((g.n, 3))
    for k in range(g.n):
        s = g.sl(k)
        M0[k] = np.sum(g.w[s, None] * dens[s], axis=0)
        M1[k] = np.sum(g.w[s, None] * np.cross(g.x[s] - g.c[k], dens[s]), axis=0)
    return M0, M1


def completion_N(g, dens, rows=None):
    """Sum_k N_k[psi]: Stokeslet (Eq. 2.19) with strength M0_k plus rotlet with
    strength M1_k, both at the centre of sphere k, at every node (Eq. 5.19);
    with `rows`, only at those nodes (other rows zero)."""
    M0, M1 = moments(g, dens)
    out = np.zeros((g.N, 3))
    x = g.x if rows is None else g.x[rows]
    acc = np.zeros((len(x), 3))
    for k in range(g.n):
        acc += kernels.stokeslet(x, g.c[k], M0[k]) + kernels.rotlet(x, g.c[k], M1[k])
    if rows is None:
        return acc
    out[rows] = acc
    return out


def rigid_part(g, dens):
    """P mu: on each sphere the rigid field F/(4 pi a^2) + (3/(8 pi a^4)) T x (x - c_k)
    with F = int mu and T = int (y - c_k) x mu, i.e. the projection of mu onto
    the translations and rotations of the sphere (P P = P for the node
    quadrature: sum w = 4 pi a^2, sum w (x - c) = 0, sum w (x-c)(x-c)^T = (4 pi a^4 / 3) I)."""
    M0, M1 = moments(g, dens)
    out = np.zeros((g.N, 3))
    for k in range(g.n):
        s = g.sl(k)
        a = g.a[k]
        out[s] = M0[k][None, :] / (4 * np.pi * a * a) + (3.0 / (8 * np.pi * a ** 4)) * np.cross(
            M1[k][None, :], g.x[s] - g.c[k])
    return out


def apply_at(g, op, dens, targets):
    """apply() restricted to the nodes of the target spheres `targets` (rows of
    other spheres are zero); used to check large problems on sampled spheres."""
    dens = np.asarray(dens, float).reshape(-1, 3)
    rows = np.concatenate([np.arange(g.sl(i).start, g.sl(i).stop) for i in targets])
    mask = np.zeros((g.N, 1))
    mask[rows] = 1.0
    if op in ("S", "D", "K"):
        return layer(g, op, dens, targets)
    if op == "mobility":
        return mask * (0.5 * dens + rigid_L(g, dens)) + layer(g, "K", dens, targets)
    if op == "resistance":
        return mask * (0.5 * dens + completion_N(g, dens, rows)) + layer(g, "D", dens, targets)
    if op == "porous":
        return mask * (0.5 * dens) + layer(g, "S", dens, targets) + layer(g, "D", dens, targets)
    if op == "squirmer":
        r = rigid_part(g, dens)
        q = dens - r
        return mask * (0.5 * q - r) + layer(g, "S", q, targets) + layer(g, "D", q, targets)
    raise ValueError(op)


def rigid_L(g, dens):
    """L_k[mu](x) = int mu + (int (y - c_k) x mu) x (x - c_k) for x on Gamma_k (Eq. 5.8)."""
    M0, M1 = moments(g, dens)
    out = np.zeros((g.N, 3))
    for k in range(g.n):
        s = g.sl(k)
        out[s] = M0[k][None, :] + np.cross(M1[k][None, :], g.x[s] - g.c[k])
    return out


def apply(g, op, dens):
    """Operators of the C interface: 'S', 'D', 'K' (raw sums), 'mobility'
    = 1/2 I + K + L (Eq. 5.8), 'resistance' = 1/2 I + D + N (Eq. 5.19),
    'porous' = 1/2 I + S + D (Eq. 5.4), and 'squirmer' = (1/2 I + S + D)(I - P) - P,
    the square form of Eq. 5.17 with the force- and torque-free conditions
    (Eq. 5.15): the rigid part P mu of the unknown carries the rigid velocity
    v_i + w_i x (x - c_i) and mu - P mu is the density (see oracle.solve)."""
    dens = np.asarray(dens, float).reshape(-1, 3)
    if op in ("S", "D", "K"):
        return layer(g, op, dens)
    if op == "mobility":
        return 0.5 * dens + layer(g, "K", dens) + rigid_L(g, dens)
    if op == "resistance":
        return 0.5 * dens + layer(g, "D", dens) + completion_N(g, dens)
    if op == "porous":
        return 0.5 * dens + layer(g, "S", dens) + layer(g, "D", dens)
    if op == "squirmer":
        r = rigid_part(g, dens)
        q = dens - r
        return 0.5 * q + layer(g, "S", q) + layer(g, "D", q) - r
    raise ValueError(op)
