"""Plain GMRES (Saad & Schultz) with modified Gram-Schmidt Arnoldi and Givens
rotations, x0 = 0, stopping on the relative l2 residual.  Test infrastructure
only.  The paper does not name its iterative solver; GMRES is the one used here.
"""
import numpy as np


def gmres(A, b, tol=1e-10, restart=200, max_iter=1000):
    """Solve A x = b.  Returns (x, info) with info = dict(iters, rel_residual
    (recomputed from b - A x), converged, history of the Arnoldi estimates)."""
    b = np.asarray(b, float).ravel()
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    hist = []
    if nb == 0.0:
        return x, dict(iters=0, rel_residual=0.0, converged=True, history=[0.0])
    total = 0
    r = b.copy()
    while True:
        beta = np.linalg.norm(r)
        m = min(restart, max_iter - total)
        if beta / nb <= tol or m <= 0:
            break
        Q = np.zeros((m + 1, len(b)))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[0] = r / beta
        k_done = 0
        for k in range(m):
            w = np.asarray(A(Q[k]), float).ravel()
            for j in range(k + 1):
                H[j, k] = np.dot(Q[j], w)
                w = w - H[j, k] * Q[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                Q[k + 1] = w / H[k + 1, k]
            for j in range(k):
                h0, h1 = H[j, k], H[j + 1, k]
                H[j, k] = cs[j] * h0 + sn[j] * h1
                H[j + 1, k] = -sn[j] * h0 + cs[j] * h1
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            total += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]) / nb)
            if abs(g[k + 1]) / nb <= tol or H[k, k] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + Q[:k_done].T @ y
        r = b - np.asarray(A(x), float).ravel()
        if total >= max_iter:
            break
    rel = np.linalg.norm(r) / nb
    return x, dict(iters=total, rel_residual=rel, converged=rel <= tol, history=hist)
