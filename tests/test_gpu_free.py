"""GPU parity of free kinematics (bodies under given force and torque, Sec. II;
body block N = (K^T M~^-1 K)^-1 in the preconditioner, Sec. VIII) against the
oracle's exact enlarged-system solution.  Tolerance as in test_gpu_solve:
solve to 1e-10, require 1e-9 on every field and on the body velocities."""
import numpy as np
import pytest

from oracle.free import FreeProblem, solve_free_fft
from oracle.system import drag
from synthetic import Body, Workload, disk_markers, small_2d, sphere_markers

from ._util import flat_fields, gpu_grid, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


def _cases():
    rng = np.random.default_rng(31)
    sph = Workload("free_sphere_32", (32, 32, 32), (1.0, 1.0, 1.0), bodies=[
        Body(np.array([0.47, 0.52, 0.5]), sphere_markers(0.2, 150), rng.standard_normal(6))])
    two = Workload("free_two_disks_64", (64, 64), (1.0, 1.0), bodies=[
        Body(np.array([0.3, 0.45]), disk_markers(0.12, 1 / 64), rng.standard_normal(3)),
        Body(np.array([0.72, 0.6]), disk_markers(0.1, 1 / 64), rng.standard_normal(3))])
    return [
        (small_2d(16, nbody=2, seed=3), [True, True]),
        (small_2d(16, nbody=2, seed=4), [True, False]),
        (two, [False, True]),
        (sph, [True]),
    ]


CASES = _cases()


def _gpu_solve(abi, wl, free, prec, tol=1e-10, UO=None):
    G = gpu_grid(abi, wl, prec, free=free)
    UO = wl.UO() if UO is None else UO
    try:
        o = abi.solve_opts_default()
        o.tol = tol
        o.max_iters = 400
        info = abi.solve_coupled(G, UO, opts=o)
        lam, ft = abi.get_forces(G, wl.d)
        U = abi.get_body_velocities(G, UO)
        n = int(np.prod(wl.n))
        v = np.zeros(wl.d * n)
        p = np.zeros(n)
        abi.get_fields(G, v, p)
    finally:
        abi.destroy_grid(G)
    return info, v, p, lam, ft, U


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_free_solve_matches_oracle(abi, case, prec):
    wl, free = CASES[case]
    fp = FreeProblem(oracle_problem(wl), free)
    vo, po, lo, Uo = solve_free_fft(fp, wl.UO())
    info, v, p, lam, ft, U = _gpu_solve(abi, wl, free, getattr(abi, prec))
    assert info.status == abi.OK, info.as_dict()
    assert rel_err(v, flat_fields(vo)) < 1e-9
    assert rel_err(p, po) < 1e-9
    assert rel_err(lam, lo) < 1e-9
    fr = np.asarray(free)
    assert rel_err(U[fr], Uo.reshape(fr.sum(), -1)) < 1e-9
    # force balance: K^T Lambda equals the applied load on each free body
    assert np.allclose(ft[fr], wl.UO()[fr], rtol=1e-8, atol=1e-10 * np.abs(wl.UO()).max())


def test_reciprocity_free_then_prescribed(abi):
    wl, free = CASES[3]
    info, v, p, lam, ft, U = _gpu_solve(abi, wl, free, abi.MIXED)
    # impose the computed velocity: the body must need exactly the applied load
    info2, v2, p2, lam2, ft2, _ = _gpu_solve(abi, wl, [False], abi.MIXED, UO=U)
    assert rel_err(ft2, wl.UO()) < 1e-8
    assert rel_err(lam2, lam) < 1e-8


def test_zero_load(abi):
    wl, _ = CASES[3]
    info, v, p, lam, ft, U = _gpu_solve(abi, wl, [True], abi.MIXED, UO=np.zeros((1, 6)))
    assert info.status == abi.OK and info.iters == 0
    assert not U.any() and not lam.any()
