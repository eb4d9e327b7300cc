"""Writes oracle_sphere128_cg.json: how many conjugate-gradient iterations the
oracle's exact Schur-complement solve (M Lambda = -(W + J v~), M = J L^-1 S~,
Sec. III.C) needs on the 128^3 periodic sphere workload (500 markers, U and
Omega ~ N(0,1), seed 1508) to reach a relative CG residual of 1e-8, and the
time of one CG iteration (one exact DFT Stokes solve with spread and
interpolation) on the machine that ran it.  Calls only oracle/ and synthetic/.

Usage: python tests/golden/make_oracle_sphere128_cg.py
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


def main():
    wl = sphere_128()
    q, rel, body = wl.markers()
    g = Grid(wl.n, wl.L, wl.eta)
    pr = Problem(g, np.mod(q, 1.0), rel, body, 1)
    W = -ib.apply_K(pr.rel, pr.body, wl.UO(), 3)
    rhs = -W.ravel()
    hist = []
    t_it = []

    def mv(x):
        t = time.time()
        f = ib.spread_tilde(g, pr.q, x.reshape(pr.N, 3))
        v, _ = fft_stokes.stokes_solve(g, f)
        out = ib.interp(g, pr.q, v).ravel()
        t_it.append(time.time() - t)
        return out

    op = spla.LinearOperator((pr.N * 3, pr.N * 3), matvec=mv, dtype=np.float64)
    # the callback only counts iterations
    lam, flag = spla.cg(op, rhs, rtol=1e-8, atol=0.0, maxiter=5000, callback=lambda xk: hist.append(0))
    iters = len(hist)
    out = {
        "workload": wl.name,
        "cg_rtol": 1e-8,
        "cg_iterations": iters,
        "cg_flag": int(flag),
        "seconds_per_iteration_median": float(np.median(t_it)),
        "cores": len(os.sched_getaffinity(0)),
        "cite": "Sec. III.C, Eqs. lambda_sol and mob_def (M is SPD: conjugate gradients)",
    }
    json.dump(out, open(os.path.join(HERE, "oracle_sphere128_cg.json"), "w"), indent=2)
    print(out)


if __name__ == "__main__":
    main()
