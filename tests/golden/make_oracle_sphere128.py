"""Writes oracle_sphere128.json: the oracle's exact solution of the 128^3
periodic sphere workload (500 markers, U and Omega ~ N(0,1), seed 1508) by
the Schur-complement route of Sec. III.C (Eqs. lambda_sol and mob_def):
conjugate gradients on M Lambda = -W with M = J L^-1 S~ (SPD), each product
one exact DFT Stokes solve, to a relative CG residual of 1e-13, then
v = L^-1 S~ Lambda.  Stored: Lambda [500][3], the body's force and torque on
the fluid K^T Lambda, and v and pi at 256 seeded cells per field (the full
fields follow from Lambda by one more exact Stokes solve).  Also records the
CG iteration count to 1e-8 and the time of one CG iteration on the machine
that ran it.  Calls only oracle/ and synthetic/.

Usage: python tests/golden/make_oracle_sphere128.py
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fft_stokes, ib  # noqa: E402
from oracle.mac import Grid  # noqa: E402
from oracle.system import Problem  # noqa: E402
from synthetic import sphere_128  # noqa: E402

SAMPLE_SEED = 128
SAMPLES = 256


def main():
    wl = sphere_128()
    q, rel, body = wl.markers()
    g = Grid(wl.n, wl.L, wl.eta)
    pr = Problem(g, np.mod(q, 1.0), rel, body, 1)
    W = -ib.apply_K(pr.rel, pr.body, wl.UO(), 3)
    rhs = -W.ravel()
    t_it = []

    def mv(x):
        t = time.time()
        f = ib.spread_tilde(g, pr.q, x.reshape(pr.N, 3))
        v, _ = fft_stokes.stokes_solve(g, f)
        out = ib.interp(g, pr.q, v).ravel()
        t_it.append(time.time() - t)
        return out

    op = spla.LinearOperator((pr.N * 3, pr.N * 3), matvec=mv, dtype=np.float64)
    res = []

    def cb(xk):
        res.append(np.linalg.norm(rhs - mv(xk)) / np.linalg.norm(rhs))

    lam, flag = spla.cg(op, rhs, rtol=1e-13, atol=0.0, maxiter=5000, callback=cb)
    it_1e8 = next(i + 1 for i, r in enumerate(res) if r <= 1e-8)
    lam = lam.reshape(pr.N, 3)
    v, p = fft_stokes.stokes_solve(g, ib.spread_tilde(g, pr.q, lam))
    rng = np.random.default_rng(SAMPLE_SEED)
    cells = rng.choice(g.ncell, size=SAMPLES, replace=False)
    out = {
        "workload": wl.name,
        "cite": "Sec. III.C, Eqs. lambda_sol and mob_def: exact Schur-complement solve, M SPD (conjugate gradients)",
        "cg_rtol": 1e-13,
        "cg_iterations": len(res),
        "cg_iterations_to_1e-8": it_1e8,
        "cg_flag": int(flag),
        "seconds_per_iteration_median": float(np.median(t_it)),
        "cores": len(os.sched_getaffinity(0)),
        "lambda": [[float(x) for x in row] for row in lam],
        "body_FT": [float(x) for x in ib.apply_KT(pr.rel, pr.body, lam, 3, 1)[0]],
        "sample_cells": [int(c) for c in cells],
        "v_samples": [[float(v[a].ravel()[c]) for c in cells] for a in range(3)],
        "p_samples": [float(p.ravel()[c]) for c in cells],
    }
    json.dump(out, open(os.path.join(HERE, "oracle_sphere128.json"), "w"), indent=1)
    print({k: out[k] for k in ("cg_iterations", "cg_iterations_to_1e-8", "cg_flag",
                               "seconds_per_iteration_median", "body_FT")})


if __name__ == "__main__":
    main()
