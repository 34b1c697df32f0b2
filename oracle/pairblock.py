"""Low-degree two-sphere interaction blocks and the pair-network reference.
Test infrastructure only.

Low modes.  A real field of VSH degree <= L on one sphere is a real vector a
of length 3(L+1)^2 - 2 (73 for L = 4): for type V (n >= 0), W, X (n >= 1), for
n, then m = 0..n: Re c_nm, and for m >= 1 also Im c_nm, where c are the complex
coefficients of oracle.vsh (field = sum_m c Z + conj).

Blocks.  For the resistance operator A = 1/2 I + D + N (Eq. 5.19) or the
mobility operator A = 1/2 I + K + L (Eq. 5.8), the block from source sphere s
to target sphere t (s != t) is B_ts = P_t A E_s, where E_s places a low-mode
field on sphere s (zero elsewhere) and P_t is the VSH analysis (Sec. 2.1) of
the result on sphere t restricted to degree <= L; the self block is B_ss.  In
the pair frame the target centre is (0, 0, d) with the source at the origin.

Network.  A fully connected net 5 -> 128 -> 128 -> 128 -> out with tanh
activations maps (pair offset in the pair frame, source radius, target radius)
to a standardised block; the reference forward / backward below are plain
FP64 numpy with the weights given (the GPU trains with BF16 weights and FP32
accumulation; tests pass it the same BF16-rounded values).
"""
import numpy as np

from . import operators as ops
from . import vsh


def low_modes(L):
    out = []
    for t in range(3):
        for n in range(L + 1):
            if t > 0 and n == 0:
                continue
            for m in range(n + 1):
                out.append((t, n, m, 0))
                if m >= 1:
                    out.append((t, n, m, 1))
    return out


def coef_to_low(c, L):
    return np.array([c[t, n, m].real if part == 0 else c[t, n, m].imag for (t, n, m, part) in low_modes(L)])


def low_to_coef(a, L, p):
    c = np.zeros((3, p + 1, p + 1), complex)
    for val, (t, n, m, part) in zip(a, low_modes(L)):
        c[t, n, m] += val if part == 0 else 1j * val
    return c


def two_sphere_blocks(centres, radii, p, L, eta=1e9, op="resistance"):
    """(B_00, B_10, B_01, B_11) of operator `op` for two spheres, probing the
    oracle operator with each low mode (all pairs treated as close for the
    default eta)."""
    g = ops.Geometry(centres, radii, p, eta=eta)
    nm = len(low_modes(L))
    B = np.zeros((2, 2, nm, nm))
    for s in range(2):
        for b in range(nm):
            dens = np.zeros((g.N, 3))
            dens[g.sl(s)] = vsh.synthesis(low_to_coef(np.eye(nm)[b], L, p))
            out = ops.apply(g, op, dens)
            for t in range(2):
                B[t, s][:, b] = coef_to_low(vsh.analysis(out[g.sl(t)], p), L)
    return B


def aligned_block(d, a_src, a_tgt, p, L, op="resistance"):
    """B_ts with the source at the origin and the target at (0, 0, d)."""
    B = two_sphere_blocks([[0.0, 0.0, 0.0], [0.0, 0.0, d]], [a_src, a_tgt], p, L, op=op)
    return B[1, 0]


# ---- reference network ------------------------------------------------------

def mlp_forward(params, X):
    """params = [W1, b1, W2, b2, W3, b3, W4, b4] (W as (in, out)); returns
    (output, cache)."""
    h = X
    cache = [X]
    for li in range(3):
        z = h @ params[2 * li] + params[2 * li + 1]
        h = np.tanh(z)
        cache.append(h)
    y = h @ params[6] + params[7]
    return y, cache


def mlp_loss_grad(params, X, Y):
    """Mean squared error over all outputs of the batch and its gradient with
    respect to every parameter (back-propagation written out)."""
    y, cache = mlp_forward(params, X)
    B, K = Y.shape
    diff = y - Y
    loss = np.sum(diff * diff) / (B * K)
    dy = 2.0 * diff / (B * K)
    grads = [None] * 8
    grads[6] = cache[3].T @ dy
    grads[7] = dy.sum(0)
    dh = dy @ params[6].T
    for li in (2, 1, 0):
        h = cache[li + 1]
        dz = dh * (1.0 - h * h)
        grads[2 * li] = cache[li].T @ dz
        grads[2 * li + 1] = dz.sum(0)
        dh = dz @ params[2 * li].T
    return loss, grads
