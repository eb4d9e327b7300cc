"""Writes oracle_bench_refs.npz: the oracle's exact solutions of the problems
whose GPU results the benchmark's batch, serving and nozzle legs report an
error for (the benchmark reads these stored values; it does not run the
oracle).  Calls only oracle/ and synthetic/.

* batch: every 64^2 and 128^2 request of the first timed batch
  (synthetic.batch_2d(64, seed=2509)): Lambda by the exact Schur route with
  the dense true mobility M = J L^-1 S~ (Sec. III.C, Eqs. lambda_sol, mob_def).
* serve: the first three 64^3 requests of the serving stream
  (synthetic.serve_3d, seed 1510; the geometry does not depend on the rate):
  Lambda by conjugate gradients on M (SPD) to a relative residual of 1e-12.
* nozzle: the 256 x 128 nozzle at Re = 0 (steady Stokes, parabolic inflow =
  outflow, no-slip channel walls; Sec. VII.F): Lambda, and v and pi at 512
  seeded cells, by the sparse LU of the whole wall-bounded system with
  iterative refinement (App. D).

Usage: python tests/golden/make_oracle_bench_refs.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fft_stokes, ib  # noqa: E402
from oracle import walls as W  # noqa: E402
from oracle.mac import Grid  # noqa: E402
from oracle.system import Problem  # noqa: E402
from synthetic import batch_2d, nozzle, parabolic_inflow, serve_3d  # noqa: E402

BATCH_SEED = 1505 + 4 + 1000
SERVE_SEED = 1505 + 5


def periodic_problem(wl):
    q, rel, body = wl.markers()
    return Problem(Grid(wl.n, wl.L, wl.eta), np.mod(q, 1.0), rel, body, len(wl.bodies))


def main():
    out = {}
    for idx, r in enumerate(batch_2d(64, seed=BATCH_SEED)):
        if r.n[0] > 128:
            continue
        wl = r.workload()
        _, _, lam = fft_stokes.solve_coupled(periodic_problem(wl), wl.UO())
        out[f"batch_{idx}_lambda"] = lam
        print("batch", idx, r.n, lam.shape, flush=True)
    got = 0
    for idx, r in enumerate(serve_3d(100, seed=SERVE_SEED)):
        if r.n[0] != 64 or got >= 3:
            continue
        wl = r.workload(ib.quat_rotate)
        _, _, lam, info = fft_stokes.solve_coupled(periodic_problem(wl), wl.UO(), dense_limit=0, cg_tol=1e-12,
                                                   return_info=True)
        out[f"serve_{idx}_lambda"] = lam
        got += 1
        print("serve", idx, r.N, info, flush=True)
    wl = nozzle(Re=0.0)
    q, rel, body = wl.markers()
    wg = W.WallGrid(wl.n, wl.L, wl.wall_flags(), wl.eta, wl.rho, wl.dt)
    prob = W.WallProblem(wg, q)
    bd = wg.zero_data()
    for s in (0, 1):
        v = np.zeros((2, wl.n[1]))
        v[0] = parabolic_inflow(wl.n[1])
        bd[(0, s)] = v.reshape(bd[(0, s)].shape)
    b = prob.rhs(-ib.apply_K(rel, body, wl.UO(), 2).ravel(), bd=bd)
    x = prob.solve(b)
    v, p, lam = prob.split(x)
    out["nozzle_re0_lambda"] = lam
    cells = np.random.default_rng(256).choice(wg.ncell, size=512, replace=False)
    out["nozzle_re0_cells"] = cells
    out["nozzle_re0_v"] = np.concatenate([a.ravel()[cells] for a in v])
    out["nozzle_re0_p"] = p.ravel()[cells]
    out["nozzle_re0_residual"] = np.array([prob.residual(x, b)])
    print("nozzle", lam.shape, prob.residual(x, b), flush=True)
    np.savez_compressed(os.path.join(HERE, "oracle_bench_refs.npz"), **out)


if __name__ == "__main__":
    main()
