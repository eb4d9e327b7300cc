"""The outer FGMRES orthogonalisations against each other, on the same solves:
classical Gram-Schmidt with reorthogonalisation over the FP64 basis,
pipelined on bulk copies (IBR_ARNOLDI=cgs2; the default below two million
entries), against modified Gram-Schmidt over the FP64 basis (=mgs; the
default from two million entries) and CGS2 over a double-float basis (=df:
pairs of floats, arithmetic on the FP32 pipe).

Every run must converge to the solve tolerance and agree with the oracle's
exact solution (and with the CGS2 run) to the accuracy that tolerance
fixes.  The orthogonalisations lose orthogonality at different rates (MGS in
proportion to the basis' condition, the double-float basis at about 2^-48
instead of 2^-53), which near a 1e-10 tolerance can cost a few outer
iterations: the counts may differ by a quarter plus two.  The cases span one
and several stages per tile sweep of the pipelined passes (k up to 8 and
beyond), a ragged last tile, restart lengths of 20 (two cycles or more), 50
and 100, 2-D and 3-D, both precisions and free bodies.
"""
import os
import pickle
import subprocess
import sys

import numpy as np
import pytest

from oracle import fft_stokes
from oracle.free import FreeProblem, solve_free_fft

from ._util import flat_fields, oracle_problem, rel_err
from synthetic import Body, Workload, disk_markers, small_2d, sphere_markers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import pickle, sys, numpy as np
sys.path.insert(0, {root!r})
import torch
from paper_1505_07865_gb300 import abi
from tests._util import gpu_grid
wl = pickle.load(open({wlfile!r}, "rb"))
G = gpu_grid(abi, wl, getattr(abi, {prec!r}), free={free!r})
o = abi.solve_opts_default()
o.tol = {tol!r}
o.restart = {restart!r}
o.max_iters = 600
info = abi.solve_coupled(G, wl.UO(), opts=o)
lam, ft = abi.get_forces(G, wl.d)
n = int(np.prod(wl.n))
v = np.zeros(wl.d * n)
p = np.zeros(n)
abi.get_fields(G, v, p)
U = abi.get_body_velocities(G, wl.UO())
np.savez({out!r}, lam=lam, v=v, p=p, U=U, iters=info.iters, status=info.status, res=info.rel_res_true)
abi.destroy_grid(G)
"""


def _solve(tmp_path, wl, prec, restart, tol, arnoldi, free=None):
    out = str(tmp_path / f"s_{arnoldi}.npz")
    env = dict(os.environ)
    env["IBR_ARNOLDI"] = arnoldi
    wlfile = str(tmp_path / "wl.pkl")
    with open(wlfile, "wb") as f:
        pickle.dump(wl, f)
    code = CHILD.format(root=ROOT, wlfile=wlfile, prec=prec, free=free, tol=tol, restart=restart, out=out)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(out))


def _cases():
    rng = np.random.default_rng(41)
    sph = Workload("sphere_32", (32, 32, 32), (1.0, 1.0, 1.0), bodies=[
        Body(np.array([0.5, 0.45, 0.52]), sphere_markers(0.2, 200), rng.standard_normal(6))])
    disks = Workload("disks_96", (96, 96), (1.0, 1.0), bodies=[
        Body(np.array([0.3, 0.4]), disk_markers(0.12, 1 / 96), rng.standard_normal(3)),
        Body(np.array([0.7, 0.62]), disk_markers(0.1, 1 / 96), rng.standard_normal(3))])
    return [("sphere32_mixed_r50", sph, "MIXED", 50, None),
            ("sphere32_mixed_r20", sph, "MIXED", 20, None),
            ("disks96_mixed_r100", disks, "MIXED", 100, None),
            ("disks96_fp64_r50", disks, "FP64", 50, None),
            ("small2d_free_mixed", small_2d(32, nbody=2, seed=7), "MIXED", 50, [True, False])]


CASES = _cases()


@pytest.mark.parametrize("alt", ["mgs", "df"])
@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_orthogonalisations_agree(tmp_path, case, alt):
    name, wl, prec, restart, free = CASES[case]
    tol = 1e-9 if restart < 50 else 1e-10
    a = _solve(tmp_path, wl, prec, restart, tol, alt, free)
    b = _solve(tmp_path, wl, prec, restart, tol, "cgs2", free)
    for r in (a, b):
        assert int(r["status"]) == 0, {k: r[k] for k in ("status", "iters", "res")}
        assert float(r["res"]) <= tol
    ia, ib = int(a["iters"]), int(b["iters"])
    assert max(ia, ib) <= 1.25 * min(ia, ib) + 2, (ia, ib)
    # both solutions agree with the oracle's exact one to what the tolerance allows
    pr = oracle_problem(wl)
    if free is None:
        vo, po, lo = fft_stokes.solve_coupled(pr, wl.UO())
        for r in (a, b):
            assert rel_err(r["lam"], lo) < 1e-8
            assert rel_err(r["v"], flat_fields(vo)) < 1e-8
    else:
        vo, po, lo, Uo = solve_free_fft(FreeProblem(pr, free), wl.UO())
        fr = np.asarray(free)
        for r in (a, b):
            assert rel_err(r["lam"], lo) < 1e-8
            assert rel_err(r["U"][fr], Uo.reshape(fr.sum(), -1)) < 1e-8
    assert rel_err(a["lam"], b["lam"]) < 1e-8


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
def test_marker_count_change_keeps_basis_pad_zero(prec):
    # a grid solved with one marker count, then with another of the other
    # parity (3-D: the system length changes parity with the marker count, so
    # the basis columns' stride and zero pad entry move): the second solve
    # must equal a fresh grid's
    from paper_1505_07865_gb300 import abi
    from tests._util import gpu_grid
    rng = np.random.default_rng(43)
    uo = rng.standard_normal(6)
    big = Workload("s1", (32, 32, 32), (1.0,) * 3, bodies=[Body(np.array([0.5, 0.5, 0.5]), sphere_markers(0.2, 200), uo)])
    small = Workload("s2", (32, 32, 32), (1.0,) * 3, bodies=[Body(np.array([0.5, 0.5, 0.5]), sphere_markers(0.18, 161), uo)])
    p = getattr(abi, prec)
    o = abi.solve_opts_default()
    o.tol = 1e-10
    G = gpu_grid(abi, big, p)
    H = gpu_grid(abi, small, p)
    try:
        assert abi.solve_coupled(G, big.UO(), opts=o).status == abi.OK
        abi.set_markers(G, 0, small.bodies[0].rel)
        i1 = abi.solve_coupled(G, small.UO(), opts=o)
        i2 = abi.solve_coupled(H, small.UO(), opts=o)
        assert i1.status == abi.OK and i2.status == abi.OK
        assert i1.iters == i2.iters
        l1, _ = abi.get_forces(G, 3)
        l2, _ = abi.get_forces(H, 3)
        assert rel_err(l1, l2) < 1e-12
    finally:
        abi.destroy_grid(G)
        abi.destroy_grid(H)
