"""Writes resistance_256_oracle_solve.json: the oracle's FP64 GMRES solve of the
256-sphere resistance workload (Problem 5, Eq. 5.19; p = 10, background shear,
spheres held fixed, tol 1e-8), its iteration and operator-apply counts, its
true residual and the forces and torques it returns.

Only oracle/ computes: oracle.solve.resistance_rhs builds the right-hand side,
oracle.gmres.gmres iterates, oracle.operators.apply_at evaluates the operator on
disjoint groups of target spheres (one worker process per host core; the groups'
rows are copied into one vector), and oracle.operators.moments gives F and T.

    python tests/golden/make_resistance_256_solve.py     (about 40 min on 8 cores)
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "resistance_256_oracle_solve.json")
GROUPS = 64

_g = None


def _init():
    global _g
    sys.path.insert(0, ROOT)
    from oracle import operators as ops
    from paper_1707_06551_gb300 import workloads as wl
    w = wl.resistance_256()
    _g = ops.Geometry(w["centres"], w["radii"], w["p"])


def _rows(g, group):
    return np.concatenate([np.arange(g.sl(i).start, g.sl(i).stop) for i in group])


def _apply_group(args):
    from oracle import operators as ops
    x, group = args
    out = ops.apply_at(_g, "resistance", x.reshape(-1, 3), group)
    return group, out[_rows(_g, group)]


def main():
    sys.path.insert(0, ROOT)
    from oracle import gmres as og
    from oracle import operators as ops
    from oracle import solve as osolve
    from paper_1707_06551_gb300 import workloads as wl
    w = wl.resistance_256()
    g = ops.Geometry(w["centres"], w["radii"], w["p"])
    groups = [list(range(i, g.n, GROUPS)) for i in range(GROUPS)]
    applies = [0]
    with mp.get_context("spawn").Pool(os.cpu_count(), initializer=_init) as pool:
        def A(x):
            applies[0] += 1
            y = np.zeros((g.N, 3))
            for group, rows in pool.map(_apply_group, [(x, q) for q in groups]):
                y[_rows(g, group)] = rows
            return y.ravel()

        b = osolve.resistance_rhs(g, w["vel"], w["omega"], w["u0"], w["G"])
        t0 = time.time()
        psi, info = og.gmres(A, b.ravel(), tol=w["tol"], restart=200, max_iter=1000)
        t1 = time.time()
    F, T = ops.moments(g, psi.reshape(-1, 3))
    rec = {"workload": "resistance_256", "p": g.p, "n_spheres": g.n, "nodes": g.N, "tol": w["tol"],
           "restart": 200, "iters": int(info["iters"]), "operator_applies": applies[0],
           "rel_residual": float(info["rel_residual"]), "converged": bool(info["converged"]),
           "history": [float(h) for h in info["history"]], "forces": F.tolist(), "torques": T.tolist(),
           "wall_s": t1 - t0, "cores": os.cpu_count()}
    with open(OUT, "w") as f:
        json.dump(rec, f)
    print(OUT, rec["iters"], rec["operator_applies"], rec["rel_residual"], rec["wall_s"])


if __name__ == "__main__":
    main()
