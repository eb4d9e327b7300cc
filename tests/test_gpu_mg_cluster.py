"""The thread-block-cluster V-cycle (periodic 3-D grids: the coarse levels in
the distributed shared memory of one 8-CTA cluster per field) against the
per-level kernels it replaces.

The same V-cycles are run in child processes with the cluster kernel forced
to start at a given level (IBR_MG_CLUSTER_LEVEL) and with IBR_MG_CLUSTER=0
(per-level kernels and the one-CTA tail); both use the same point arithmetic
and sweep order, so they agree to rounding (1e-13 relative in FP64, 1e-6 in
FP32; in practice bitwise).  Convergence to the exact DFT solution is checked
by test_gpu_ops.py's V-cycle test, and the schedule autotuner's choice here.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# (grid, sigma, precision, first cluster level)
CASES = [((64, 64, 64), 0.0, "FP64", 1), ((64, 64, 64), 2e3, "MIXED", 0), ((128, 128, 128), 0.0, "MIXED", 1),
         ((128, 128, 128), 0.0, "MIXED", 2), ((96, 64, 64), 0.0, "FP64", 1), ((48, 48, 48), 5e2, "FP64", 0),
         ((192, 192, 192), 0.0, "MIXED", 2), ((32, 32, 32), 0.0, "MIXED", 0)]

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1505_07865_gb300 import abi
n, sigma, prec, out = {n!r}, {sigma!r}, {prec!r}, {out!r}
d = len(n)
L = [v / n[0] for v in n]
G = abi.create_grid(d, n, L, precision=getattr(abi, prec))
rng = np.random.default_rng(5)
ncell = int(np.prod(n))
f = rng.standard_normal(ncell)
if sigma == 0.0:
    f -= f.mean()
u = torch.tensor(rng.standard_normal(ncell), device="cuda")
abi.op_vcycle(G, sigma, 1.3, torch.tensor(f, device="cuda"), u, 2)
torch.cuda.synchronize()
np.save(out, u.cpu().numpy())
abi.destroy_grid(G)
"""


def _run(tmp_path, n, sigma, prec, level):
    out = str(tmp_path / f"u_{level}.npy")
    env = dict(os.environ)
    if level is None:
        env["IBR_MG_CLUSTER"] = "0"
    else:
        env["IBR_MG_CLUSTER_LEVEL"] = str(level)
    code = CHILD.format(root=ROOT, n=n, sigma=sigma, prec=prec, out=out)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


@pytest.mark.parametrize("n,sigma,prec,level", CASES,
                         ids=[f"{'x'.join(map(str, c[0]))}_{c[2]}_s{c[1]:g}_L{c[3]}" for c in CASES])
def test_cluster_vcycle_equals_per_level_kernels(tmp_path, n, sigma, prec, level):
    uc = _run(tmp_path, n, sigma, prec, level)
    up = _run(tmp_path, n, sigma, prec, None)
    err = np.linalg.norm(uc - up) / np.linalg.norm(up)
    print(n, prec, sigma, level, err)
    assert err < (1e-13 if prec == "FP64" else 1e-6), err


def test_schedule_autotuner_picks_a_candidate():
    # a 64^3 solve's multigrid set-up times the schedules of its hierarchy
    # (velocity: 3 stacked fields, pressure: 1) and keeps one of them
    from paper_1505_07865_gb300 import abi
    from synthetic import Body, Workload, sphere_markers

    from ._util import gpu_grid

    wl = Workload("tune_cl", (64, 64, 64), (1.0, 1.0, 1.0),
                  bodies=[Body(np.array([0.5, 0.5, 0.5]), sphere_markers(0.2, 120), np.ones(6))], tol=1e-8)
    G = gpu_grid(abi, wl, abi.MIXED)
    try:
        abi.solve_coupled(G, wl.UO(), opts=abi.solve_opts_default())
    finally:
        abi.destroy_grid(G)
    mine = [t for t in abi.tuned_vcycle_schedules() if t[:3] == (64, 64, 64) and t[5] == 4]
    assert {t[4] for t in mine} == {1, 3}, mine
    for t in mine:
        assert t[6] in (-2, 0, 1), t


PS_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1505_07865_gb300 import abi
n, prec, out = {n!r}, {prec!r}, {out!r}
G = abi.create_grid(3, n, [v / n[0] for v in n], precision=getattr(abi, prec))
ncell = int(np.prod(n))
r = torch.tensor(np.random.default_rng(3).standard_normal(4 * ncell), device="cuda")
z = torch.zeros(4 * ncell, dtype=torch.float64, device="cuda")
abi.op_stokes_pc(G, r, z)
torch.cuda.synchronize()
np.save(out, z.cpu().numpy())
abi.destroy_grid(G)
"""


@pytest.mark.parametrize("n,prec", [((64, 48, 32), "MIXED"), ((128, 128, 128), "MIXED"), ((64, 64, 64), "FP64"),
                                    ((96, 96, 96), "MIXED")])
def test_split_layout_finest_level_equals_natural(tmp_path, n, prec):
    # one application of P_S (its zero-start V-cycles run the finest level and
    # level 1 in red-black split layout) against the same with IBR_MG_SPLIT=0
    outs = []
    for split in ("1", "0"):
        out = str(tmp_path / f"z_{split}.npy")
        env = dict(os.environ)
        env["IBR_MG_SPLIT"] = split
        code = PS_CHILD.format(root=ROOT, n=n, prec=prec, out=out)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        outs.append(np.load(out))
    err = np.linalg.norm(outs[0] - outs[1]) / np.linalg.norm(outs[1])
    print(n, prec, err)
    assert err < (1e-13 if prec == "FP64" else 1e-6), err
