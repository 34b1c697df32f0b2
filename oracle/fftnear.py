"""FFT-accelerated close-pair evaluation with rotations (Sec. 4.2, Fig. 2).
Test infrastructure only.

For a close source sphere k and target sphere i the paper evaluates the source's
exterior expansion in a frame whose pole points from c_k to c_i:

  (1) density rotation: the source density's VSH coefficients in the rotated
      frame (a rotation keeps the degree, so they are exact);
  (2) evaluation on the target grid aligned with the rotated pole: the target
      sphere's grid of Eq. 4.2 placed about the target centre in the rotated
      frame -- its nodes then lie on p+1 discs about the pole, at constant
      (r, theta) and equispaced phi, which is what makes the evaluation an
      FFT in phi on the GPU; the oracle evaluates the exterior formulas
      (Eqs. 3.6-3.11, traction of Eq. 3.18 with the target normals) there
      directly;
  (3) function-sample rotation: the samples, a vector field on the target
      sphere in the rotated frame, are analysed on that grid (a forward VSH
      transform), the coefficients rotated back to the original frame, and
      the field synthesised at the original target nodes.

Stage (3) projects the close-pair field onto VSH degree <= p on the target
sphere, so the result is a different discrete operator from the direct
evaluation at the nodes (oracle.operators.near_term), converging to it
spectrally in p.

The rotated frame (reading of the paper, which leaves it open): with
(sin b cos a, sin b sin a, cos b) the unit vector from c_k to c_i, the frame
x' = Q x has Q^T = R_z(a) R_y(b) (so Q^T e_z is that vector); on the polar axis
(b = 0 or pi) a = 0.
"""
import numpy as np

from . import offsurface, operators as ops, vsh
from .offsurface import _rotated_coeffs


def rot_z(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(t):
    c, s = np.cos(t), np.sin(t)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def pair_frame(c_src, c_tgt):
    """(Q, d): the rotation to the frame whose pole points from c_src to c_tgt
    (x' = Q x, Q^T = R_z(a) R_y(b)) and the centre distance d."""
    v = np.asarray(c_tgt, float) - np.asarray(c_src, float)
    d = np.linalg.norm(v)
    b = np.arccos(np.clip(v[2] / d, -1.0, 1.0))
    a = np.arctan2(v[1], v[0]) if np.hypot(v[0], v[1]) > 0 else 0.0
    Qt = rot_z(a) @ rot_y(b)
    return Qt.T, d


def near_pair(op, coef_src, a_src, c_src, c_tgt, a_tgt, p):
    """Contribution of source sphere (coefficients coef_src of its density on
    the unit sphere, radius a_src, centre c_src) to the nodes of a target
    sphere (centre c_tgt, radius a_tgt, grid of order p) by stages (1)-(3).
    op: 'S', 'D' or 'K' (traction with the target's outward normals)."""
    Q, d = pair_frame(c_src, c_tgt)
    cr = _rotated_coeffs(coef_src, Q)                       # (1)
    ct, st, cp, sp = vsh.grid_angles(p)
    dirs = np.stack([st * cp, st * sp, ct], axis=-1).reshape(-1, 3)
    xh = np.array([0.0, 0.0, d / a_src])[None, :] + (a_tgt / a_src) * dirs
    if op == "S":                                            # (2)
        u = a_src * offsurface.S_velocity(cr, xh)
    elif op == "D":
        u = offsurface.D_velocity(cr, xh)
    elif op == "K":
        u = offsurface.S_traction(cr, xh, dirs)
    else:
        raise ValueError(op)
    cu = vsh.analysis(u, p)                                  # (3)
    return vsh.synthesis(_rotated_coeffs(cu, Q.T))


def near_term(g, op, dens, coefs=None, targets=None):
    """Sum over close pairs of near_pair (the FFT-accelerated counterpart of
    oracle.operators.near_term)."""
    coefs = ops.coefficients(g, dens) if coefs is None else coefs
    out = np.zeros_like(np.asarray(dens, float).reshape(-1, 3))
    tg = range(g.n) if targets is None else list(targets)
    for i in tg:
        for k in g.near[i]:
            out[g.sl(i)] += near_pair(op, coefs[k], g.a[k], g.c[k], g.c[i], g.a[i], g.p)
    return out


def layer(g, op, dens, targets=None):
    """Raw layer sum with the close pairs by the rotated scheme."""
    dens = np.asarray(dens, float).reshape(-1, 3)
    coefs = ops.coefficients(g, dens)
    return (ops.self_term(g, op, dens, coefs, targets) + ops.far_term(g, op, dens, targets)
            + near_term(g, op, dens, coefs, targets))


def apply(g, op, dens, targets=None):
    """The operators of oracle.operators.apply / apply_at (S, D, K, mobility,
    resistance, porous, squirmer) with the rotated close-pair scheme (rows of
    other spheres zero when targets are given)."""
    dens = np.asarray(dens, float).reshape(-1, 3)
    rows = np.arange(g.N) if targets is None else np.concatenate(
        [np.arange(g.sl(i).start, g.sl(i).stop) for i in targets])
    mask = np.zeros((g.N, 1))
    mask[rows] = 1.0
    if op in ("S", "D", "K"):
        return layer(g, op, dens, targets)
    if op == "mobility":
        return mask * (0.5 * dens + ops.rigid_L(g, dens)) + layer(g, "K", dens, targets)
    if op == "resistance":
        return mask * (0.5 * dens + ops.completion_N(g, dens, rows)) + layer(g, "D", dens, targets)
    if op == "porous":
        return mask * (0.5 * dens) + layer(g, "S", dens, targets) + layer(g, "D", dens, targets)
    if op == "squirmer":
        r = ops.rigid_part(g, dens)
        q = dens - r
        return mask * (0.5 * q - r) + layer(g, "S", q, targets) + layer(g, "D", q, targets)
    raise ValueError(op)
