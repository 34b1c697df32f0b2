"""Seeded synthetic suspensions (sphere placements, forces, background flows).

This module holds geometry and random draws only -- none of the method's
arithmetic -- so that the CUDA path and the CPU oracle can be fed identical
inputs.  All randomness comes from numpy.random.default_rng(seed).

Workloads (the paper uses no public data set):
  mobility_8      8 unit spheres, centres uniform in [0, 12]^3 with minimum
                  centre distance 2.5, F, T ~ N(0, 1), p = 6.
  resistance_256  256 unit spheres, random sequential addition at volume
                  fraction 0.10 in a cube, then 20% of the spheres moved towards
                  their nearest neighbour to a surface gap ~ U[0.05, 0.2];
                  p = 10; background shear u_inf = (y, 0, 0); spheres held fixed.
  batched_512     512 independent mobility problems with n ~ U{4..64},
                  p ~ U{6, 8, 10, 12}, radii log-uniform in [0.5, 2], RSA at
                  volume fraction 0.05 with minimum gap 0.1 (a_i + a_k).
  dense_1024      1024 unit spheres, RSA at volume fraction 0.30, nearest gap of
                  each sphere pushed to log-uniform [0.01, 0.5], p = 12.
  large_4096      4096 spheres, radii ~ U[0.8, 1.2], RSA at volume fraction
                  0.20, p = 12, resistance in a random linear flow u0 + G x
                  (G traceless).
"""
import math

import numpy as np


class _Cells:
    """Uniform cell list for overlap queries during placement."""

    def __init__(self, L, h):
        self.h = h
        self.n = max(1, int(math.ceil(L / h)))
        self.cells = {}

    def key(self, x):
        return tuple(np.clip((np.asarray(x) // self.h).astype(int), -1, self.n))

    def add(self, idx, x):
        self.cells.setdefault(self.key(x), []).append(idx)

    def remove(self, idx, x):
        self.cells[self.key(x)].remove(idx)

    def around(self, x):
        k = self.key(x)
        out = []
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    out.extend(self.cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ()))
        return out


def rsa(rng, radii, L, min_gap_fn=lambda ai, ak: 0.0, max_tries=2_000_000):
    """Random sequential addition of spheres with the given radii, centres
    uniform in [0, L]^3, rejecting any draw closer than min_gap_fn to a placed
    sphere.  Radii are placed in the given order."""
    radii = np.asarray(radii, float)
    amax = float(np.max(radii))
    cells = _Cells(L, 2.0 * amax + min_gap_fn(amax, amax) + 1e-9)
    c = np.zeros((len(radii), 3))
    tries = 0
    for i, a in enumerate(radii):
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("placement failed; volume fraction too high")
            x = rng.uniform(0.0, L, size=3)
            ok = True
            for k in cells.around(x):
                if np.linalg.norm(x - c[k]) - a - radii[k] < min_gap_fn(a, radii[k]):
                    ok = False
                    break
            if ok:
                c[i] = x
                cells.add(i, x)
                break
    return c


def push_gaps(rng, c, radii, frac, gap_sampler, min_gap, L):
    """Move a fraction of spheres along the line to their nearest neighbour so
    that their surface gap becomes gap_sampler(); moves that would bring any
    other pair below min_gap are rejected (the sphere then stays put)."""
    c = c.copy()
    n = len(radii)
    chosen = rng.choice(n, size=int(round(frac * n)), replace=False)
    for i in chosen:
        d = np.linalg.norm(c - c[i], axis=1) - radii - radii[i]
        d[i] = np.inf
        j = int(np.argmin(d))
        g = gap_sampler()
        u = c[i] - c[j]
        u /= np.linalg.norm(u)
        x = c[j] + u * (radii[i] + radii[j] + g)
        dd = np.linalg.norm(c - x, axis=1) - radii - radii[i]
        dd[i] = np.inf
        dd[j] = np.inf
        if np.all(dd >= min_gap):
            c[i] = x
    return c


def mobility_8(seed=0):
    rng = np.random.default_rng(seed)
    radii = np.ones(8)
    c = rsa(rng, radii, 12.0, lambda ai, ak: 0.5)
    F = rng.normal(size=(8, 3))
    T = rng.normal(size=(8, 3))
    return dict(name="mobility_8", centres=c, radii=radii, p=6, forces=F, torques=T, tol=1e-10)


def resistance_256(seed=1):
    rng = np.random.default_rng(seed)
    n = 256
    radii = np.ones(n)
    L = (n * 4.0 / 3.0 * math.pi / 0.10) ** (1.0 / 3.0)
    c = rsa(rng, radii, L, lambda ai, ak: 0.05)
    c = push_gaps(rng, c, radii, 0.20, lambda: rng.uniform(0.05, 0.2), 0.05, L)
    G = np.zeros((3, 3))
    G[0, 1] = 1.0
    return dict(name="resistance_256", centres=c, radii=radii, p=10, vel=np.zeros((n, 3)),
                omega=np.zeros((n, 3)), u0=np.zeros(3), G=G, tol=1e-8)


def small_suspension(n, p, seed, box=None, radius_range=(1.0, 1.0), min_gap=0.05, push=0.3,
                     gap_range=(0.05, 0.3)):
    """A small random suspension for parity tests: RSA in a cube sized for a
    volume fraction near 0.1, then a fraction `push` of spheres moved to gaps
    U[gap_range] so that near pairs exist."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(radius_range[0], radius_range[1], size=n)
    if box is None:
        box = (np.sum(4.0 / 3.0 * math.pi * radii ** 3) / 0.10) ** (1.0 / 3.0) + 2.0
    c = rsa(rng, radii, box, lambda ai, ak: min_gap)
    if push > 0:
        c = push_gaps(rng, c, radii, push, lambda: rng.uniform(*gap_range), min_gap, box)
    return dict(centres=c, radii=radii, p=p)


def batched_512(seed=2, n_problems=512):
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(n_problems):
        n = int(rng.integers(4, 65))
        p = int(rng.choice([6, 8, 10, 12]))
        radii = np.exp(rng.uniform(math.log(0.5), math.log(2.0), size=n))
        L = (np.sum(4.0 / 3.0 * math.pi * radii ** 3) / 0.05) ** (1.0 / 3.0)
        c = rsa(rng, radii, L, lambda ai, ak: 0.1 * (ai + ak))
        probs.append(dict(centres=c, radii=radii, p=p, forces=rng.normal(size=(n, 3)),
                          torques=rng.normal(size=(n, 3))))
    return probs


def dense_1024(seed=3):
    rng = np.random.default_rng(seed)
    n = 1024
    radii = np.ones(n)
    L = (n * 4.0 / 3.0 * math.pi / 0.30) ** (1.0 / 3.0)
    c = rsa(rng, radii, L, lambda ai, ak: 0.01)
    c = push_gaps(rng, c, radii, 1.0, lambda: math.exp(rng.uniform(math.log(0.01), math.log(0.5))), 0.01, L)
    return dict(name="dense_1024", centres=c, radii=radii, p=12, forces=rng.normal(size=(n, 3)),
                torques=rng.normal(size=(n, 3)))


def large_4096(seed=4):
    rng = np.random.default_rng(seed)
    n = 4096
    radii = rng.uniform(0.8, 1.2, size=n)
    L = (np.sum(4.0 / 3.0 * math.pi * radii ** 3) / 0.20) ** (1.0 / 3.0)
    c = rsa(rng, radii, L, lambda ai, ak: 0.01)
    G = rng.normal(size=(3, 3))
    G -= np.trace(G) / 3.0 * np.eye(3)
    return dict(name="large_4096", centres=c, radii=radii, p=12, vel=np.zeros((n, 3)),
                omega=np.zeros((n, 3)), u0=rng.normal(size=3), G=G)


def squirmer_slip(normals, axes, B1, B2):
    """Tangential squirmer slip at surface nodes with outward unit normals n:
    u_s = (B1 + B2 cos t) sin t e_t, t the polar angle from the swimming axis e
    of the node's sphere; with sin t e_t = (n . e) n - e this is
    u_s = (B1 + B2 (n . e)) ((n . e) n - e).  `axes` holds
    the axis e of each node's sphere ([N][3]); B1, B2 per node (scalars or
    [N] arrays).  B2 > 0 is a puller, B2 < 0 a pusher."""
    n = np.asarray(normals, float).reshape(-1, 3)
    e = np.asarray(axes, float).reshape(-1, 3)
    ne = np.sum(n * e, axis=1)
    return ((np.asarray(B1, float) + np.asarray(B2, float) * ne)[:, None]) * (ne[:, None] * n - e)


def smooth_density(nodes, centres, npn, seed, modes=4, k_max=1.0):
    """A smooth nodal vector field for operator applies: per sphere a random
    rigid motion v + w x (x - c) (unit-variance components), plus `modes`
    plane waves a sin(k . x + phi) with |k| <= k_max and unit-variance
    amplitudes a.  `nodes` [N][3] in sphere order (npn nodes per sphere),
    `centres` [n][3]."""
    rng = np.random.default_rng(seed)
    x = np.asarray(nodes, float).reshape(-1, 3)
    c = np.asarray(centres, float).reshape(-1, 3)
    n = len(c)
    v, w = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    r = x.reshape(n, npn, 3) - c[:, None, :]
    u = (v[:, None, :] + np.cross(np.broadcast_to(w[:, None, :], r.shape), r)).reshape(-1, 3)
    for _ in range(modes):
        k = rng.normal(size=3)
        k *= k_max * rng.uniform() / np.linalg.norm(k)
        u = u + rng.normal(size=3)[None, :] * np.sin(x @ k + rng.uniform(0, 2 * np.pi))[:, None]
    return u


def squirmers(n, p, seed, B1=1.0, beta=-3.0, radius_range=(1.0, 1.0)):
    """A small suspension of squirmers (RSA at volume fraction near 0.1, some
    pairs pushed close) with random unit swimming axes; B2 = beta B1
    (beta < 0: pushers)."""
    w = small_suspension(n, p, seed, radius_range=radius_range)
    rng = np.random.default_rng(seed + 1000)
    ax = rng.normal(size=(n, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    w.update(axes=ax, B1=B1, B2=beta * B1)
    return w


def lattice(m, q, poly=False):
    """Cubic lattice of the operator-apply scaling tests (Sec. 6): m x m x m
    unit cubes of side 2 with a sphere of radius r_v = 1 - 2^-q on every vertex
    ((m+1)^3 spheres: 8, 27, 125, 729, 4913 for m = 1, 2, 4, 8, 16); minimum gap
    2^(1-q).  poly=True adds a sphere at the centre of every face and one at
    the centre of every cube (n = (m+1)^3 + 3 m^2 (m+1) + m^3: 15, 71, 429,
    2969, 22065).  The face and centre radii are those of the holes of the
    vertex packing scaled by r_v: r_f = (sqrt 2 - 1) r_v and
    r_c = (2 - sqrt 2) r_v (as printed, (2 - sqrt 2) r_v on the faces would
    overlap the vertex spheres at q = 4); the minimum gap is then 2^-q
    (centre sphere to face sphere)."""
    rv = 1.0 - 2.0 ** (-q)
    g = np.arange(m + 1) * 2.0
    cs = [np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)]
    rs = [np.full(len(cs[0]), rv)]
    if poly:
        h = np.arange(m) * 2.0 + 1.0
        faces = []
        for ax in range(3):
            # faces normal to axis ax: coordinate ax on the lattice planes, the others at cube centres
            grids = [h, h, h]
            grids[ax] = g
            faces.append(np.stack(np.meshgrid(*grids, indexing="ij"), axis=-1).reshape(-1, 3))
        faces = np.concatenate(faces)
        cs.append(faces)
        rs.append(np.full(len(faces), (math.sqrt(2.0) - 1.0) * rv))
        cent = np.stack(np.meshgrid(h, h, h, indexing="ij"), axis=-1).reshape(-1, 3)
        cs.append(cent)
        rs.append(np.full(len(cent), (2.0 - math.sqrt(2.0)) * rv))
    return dict(name=f"lattice_m{m}_q{q}_{'poly' if poly else 'mono'}", centres=np.concatenate(cs),
                radii=np.concatenate(rs), m=m, q=q, poly=poly)
