"""Eigenvalues ("signatures") of the Stokes boundary integral operators on the
unit sphere, Theorem 2 (Eq. 3.12).  Test infrastructure only.

Rows S, D+, D-, K+, K-; columns V, W, X.  '+' is the exterior limit (the r > 1
branches of Eqs. 3.6-3.11 at r = 1), '-' the interior one.
"""


def S(n):
    return (n / ((2 * n + 1) * (2 * n + 3)), (n + 1) / ((2 * n + 1) * (2 * n - 1)), 1.0 / (2 * n + 1))


def D_plus(n):
    return ((2 * n * n + 4 * n + 3) / ((2 * n + 1) * (2 * n + 3)),
            2 * (n - 1) * (n + 1) / ((2 * n + 1) * (2 * n - 1)),
            (n - 1) / (2 * n + 1))


def D_minus(n):
    return (-2 * n * (n + 2) / ((2 * n + 1) * (2 * n + 3)),
            -(2 * n * n + 1) / ((2 * n + 1) * (2 * n - 1)),
            -(n + 2) / (2 * n + 1))


def K_plus(n):
    return D_minus(n)


def K_minus(n):
    return D_plus(n)


def D_pv(n):
    """On-surface principal value (D+ + D-)/2; the self-interaction of the
    discrete D and K operators.  Then 1/2 + D_pv = D+ (Eqs. 5.4, 5.19) and
    1/2 + K_pv = K- (Eq. 5.8), with K_pv = D_pv since K+ = D- and K- = D+."""
    a, b = D_plus(n), D_minus(n)
    return tuple(0.5 * (x + y) for x, y in zip(a, b))


def K_pv(n):
    a, b = K_plus(n), K_minus(n)
    return tuple(0.5 * (x + y) for x, y in zip(a, b))
