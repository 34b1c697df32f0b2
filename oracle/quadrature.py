"""Sphere grid and smooth quadrature (Sec. 4, Eqs. 4.2-4.4).  Test infrastructure only."""
import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (Sec. 4, Eq. 4.2).

    Nodes are the roots of P_n, found by Newton iteration with P_n and P_n'
    from the three-term Legendre recurrence.  Returned in DESCENDING order of
    t, so that theta = arccos(t) ascends from the north pole.
    Weights: lambda = 2 / ((1 - t^2) P_n'(t)^2).
    """
    if n < 1:
        raise ValueError("n >= 1 required")
    t = np.cos(np.pi * (np.arange(1, n + 1) - 0.25) / (n + 0.5))
    for _ in range(200):
        p_prev = np.ones_like(t)
        p_cur = t.copy()
        for k in range(2, n + 1):
            p_prev, p_cur = p_cur, ((2 * k - 1) * t * p_cur - (k - 1) * p_prev) / k
        dp = n * (t * p_cur - p_prev) / (t * t - 1.0)
        step = p_cur / dp
        t = t - step
        if np.max(np.abs(step)) < 1e-15:
            break
    p_prev = np.ones_like(t)
    p_cur = t.copy()
    for k in range(2, n + 1):
        p_prev, p_cur = p_cur, ((2 * k - 1) * t * p_cur - (k - 1) * p_prev) / k
    dp = n * (t * p_cur - p_prev) / (t * t - 1.0)
    lam = 2.0 / ((1.0 - t * t) * dp * dp)
    return t, lam


def grid(p):
    """Parametric grid of Eq. 4.2: theta_j = arccos(t_j), j = 0..p (t_j the
    (p+1)-point Gauss-Legendre nodes) and phi_k = 2 pi k / (2p+2), k = 0..2p+1.

    Returns (t, lam, theta, phi)."""
    t, lam = gauss_legendre(p + 1)
    theta = np.arccos(t)
    phi = 2.0 * np.pi * np.arange(2 * p + 2) / (2 * p + 2)
    return t, lam, theta, phi


def unit_weights(p):
    """Smooth-quadrature weights on the UNIT sphere per grid node (Eq. 4.4 with
    the area element W = sin(theta)): 2 pi lambda_j / (2p+2), shape (p+1, 2p+2)."""
    t, lam, theta, phi = grid(p)
    w = 2.0 * np.pi * lam / (2 * p + 2)
    return np.repeat(w[:, None], 2 * p + 2, axis=1)


def sphere_nodes(centre, radius, p):
    """Quadrature nodes, outward normals and weights of one sphere (Eqs. 4.2, 4.4).

    x_jk = c + a e_r(theta_j, phi_k); n = e_r; weight = 2 pi a^2 lambda_j / (2p+2)
    (area element W = a^2 sin(theta) cancels the 1/sin(theta) of Eq. 4.4).
    Node order: latitude j major, longitude k minor.  Returns arrays of shape
    (nodes, 3), (nodes, 3), (nodes,)."""
    t, lam, theta, phi = grid(p)
    st = np.sqrt(1.0 - t * t)
    er = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)),
                   np.outer(t, np.ones_like(phi))], axis=-1).reshape(-1, 3)
    x = np.asarray(centre, float)[None, :] + radius * er
    w = np.repeat(2.0 * np.pi * radius * radius * lam / (2 * p + 2), 2 * p + 2)
    return x, er, w
