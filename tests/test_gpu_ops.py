"""GPU parity of each step of the hot path against the FP64 oracle, through
the C ABI (FP64 entry points).

Tolerances: the FP64 kernels evaluate the same sums as the oracle in another
order, so agreement is at rounding level; 1e-12 relative (the sums have at
most ~10^2 terms of one sign pattern each) is used throughout.
"""
import numpy as np
import pytest

from oracle import fft_stokes, ib, mobility
from oracle.mac import Grid
from synthetic import Body, Workload, disk_markers, small_2d, small_3d, sphere_128, sphere_markers

from ._util import gpu_grid, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


def _cases():
    rng = np.random.default_rng(3)
    two = Workload("two_disks_96x64", (96, 64), (1.5, 1.0), bodies=[
        Body(np.array([0.37, 0.41]), disk_markers(0.12, 1 / 64), rng.standard_normal(3)),
        Body(np.array([1.13, 0.62]), disk_markers(0.08, 1 / 64), rng.standard_normal(3)),
    ])
    seam = Workload("disk_on_seam_32", (32, 32), (1.0, 1.0), bodies=[
        Body(np.array([0.01, 0.985]), disk_markers(0.1, 1 / 32), rng.standard_normal(3))])
    sph = Workload("sphere_40x32x24", (40, 32, 24), (1.25, 1.0, 0.75), bodies=[
        Body(np.array([0.61, 0.52, 0.37]), sphere_markers(0.15, 90), rng.standard_normal(6))])
    return [small_2d(16), two, seam, small_3d(8), sph]


CASES = _cases()
IDS = [c.name for c in CASES]


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_spread_interp_rigid_parity(abi, wl):
    pr = oracle_problem(wl)
    g = pr.grid
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        abi.prepare(G)
        rng = np.random.default_rng(11)
        lam = rng.standard_normal((pr.N, g.d))
        v = [rng.standard_normal(g.shape) for _ in range(g.d)]
        f_dev = torch.zeros(g.d * g.ncell, dtype=torch.float64, device="cuda")
        abi.op_spread(G, _t(lam), f_dev)
        f_or = np.concatenate([a.ravel() for a in ib.spread_tilde(g, pr.q, lam)])
        assert rel_err(f_dev.cpu().numpy(), f_or) < TOL
        U_dev = torch.zeros(pr.N * g.d, dtype=torch.float64, device="cuda")
        abi.op_interp(G, _t(np.concatenate([a.ravel() for a in v])), U_dev)
        assert rel_err(U_dev.cpu().numpy(), ib.interp(g, pr.q, v)) < TOL
        UO = rng.standard_normal((len(wl.bodies), g.d + (1 if g.d == 2 else 3)))
        V_dev = torch.zeros(pr.N * g.d, dtype=torch.float64, device="cuda")
        abi.op_rigid(G, _t(UO), V_dev)
        assert rel_err(V_dev.cpu().numpy(), ib.apply_K(pr.rel, pr.body, UO, g.d)) < TOL
        FT_dev = torch.zeros(UO.size, dtype=torch.float64, device="cuda")
        abi.op_rigid_T(G, _t(lam), FT_dev)
        assert rel_err(FT_dev.cpu().numpy(), ib.apply_KT(pr.rel, pr.body, lam, g.d, len(wl.bodies))) < TOL
    finally:
        abi.destroy_grid(G)


@pytest.mark.parametrize("wl", CASES + [small_2d(16, rho=1.0, dt=1e-3)], ids=IDS + ["unsteady2d"])
def test_system_matvec_parity(abi, wl):
    pr = oracle_problem(wl)
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        abi.prepare(G)
        rng = np.random.default_rng(12)
        x = rng.standard_normal(pr.size)
        y_dev = torch.zeros(pr.size, dtype=torch.float64, device="cuda")
        abi.apply_system(G, _t(x), y_dev)
        assert rel_err(y_dev.cpu().numpy(), pr.matvec(x)) < TOL
    finally:
        abi.destroy_grid(G)


def test_spread_gather_is_deterministic(abi):
    wl = sphere_128()
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        abi.prepare(G)
        N = wl.bodies[0].rel.shape[0]
        lam = _t(np.random.default_rng(1).standard_normal(3 * N))
        outs = []
        for _ in range(3):
            f = torch.zeros(3 * 128 ** 3, dtype=torch.float64, device="cuda")
            abi.op_spread(G, lam, f)
            outs.append(f)
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    finally:
        abi.destroy_grid(G)


def test_mtilde_build_parity_3d_rpy(abi):
    wl = sphere_128()
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        abi.prepare(G)
        rel = wl.bodies[0].rel
        n = rel.size
        out = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, out)
        ref = mobility.mtilde_3d_rpy(rel, 1.0 / 128, 1.0, 1.0, 1.25, periodic=True)
        assert rel_err(out.cpu().numpy(), ref) < TOL
    finally:
        abi.destroy_grid(G)


def test_mtilde_build_parity_2d_form(abi):
    wl = small_2d(64, radius_h=6.4)
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        o = abi.solve_opts_default()
        abi.prepare(G, o)
        rel = wl.bodies[0].rel
        n = rel.size
        out = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, out)
        aoh, coef = abi.mobility_defaults(2)
        ref = mobility.mtilde_2d_steady(rel, 1.0 / 64, 1.0, 1.0, aoh, list(coef))
        assert rel_err(out.cpu().numpy(), ref) < TOL
    finally:
        abi.destroy_grid(G)


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-9), ("MIXED", 1e-3)])
def test_mtilde_solve_inverts(abi, prec, tol):
    wl = sphere_128()
    G = gpu_grid(abi, wl, getattr(abi, prec))
    try:
        abi.prepare(G)
        rel = wl.bodies[0].rel
        n = rel.size
        M = mobility.mtilde_3d_rpy(rel, 1.0 / 128, 1.0, 1.0, 1.25, periodic=True)
        x = np.random.default_rng(2).standard_normal(n)
        out = torch.zeros(n, dtype=torch.float64, device="cuda")
        abi.op_mtilde_solve(G, _t(M @ x), out)
        kappa = np.linalg.cond(M)
        assert rel_err(out.cpu().numpy(), x) < tol * max(1.0, kappa / 1e3)
    finally:
        abi.destroy_grid(G)


@pytest.mark.parametrize("n,sigma", [((64, 64), 0.0), ((48, 32), 5e3), ((32, 32, 32), 0.0), ((24, 16, 32), 1e4),
                                     ((96, 64, 64), 0.0)])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_vcycle_converges_to_exact_solution(abi, n, sigma, prec):
    # (96, 64, 64): a level large enough for the smoother's tile autotuner
    d = len(n)
    L = [v / n[0] for v in n]
    wl = Workload("mg", n, tuple(L), bodies=[Body(np.array(L) * 0.5, np.zeros((1, d)) + 0.01, np.zeros(d + (1 if d == 2 else 3)))])
    g = Grid(n, L)
    G = gpu_grid(abi, wl, getattr(abi, prec))
    try:
        rng = np.random.default_rng(5)
        f = rng.standard_normal(g.shape)
        if sigma == 0.0:
            f -= f.mean()
        kappa = 1.3
        exact = fft_stokes.helmholtz_solve(g, sigma, kappa, f)
        u = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
        errs = []
        for _ in range(8):
            abi.op_vcycle(G, sigma, kappa, _t(f), u, 1)
            un = u.cpu().numpy().reshape(g.shape)
            if sigma == 0.0:
                un = un - un.mean()
            errs.append(rel_err(un, exact))
        rate = (errs[5] / errs[0]) ** (1 / 5)
        floor = 1e-12 if prec == "FP64" else 1e-5
        assert errs[-1] < max(floor, 1e-6) or rate < 0.25, (errs, rate)
        assert rate < 0.35 or errs[-1] < floor * 10, (errs, rate)
    finally:
        abi.destroy_grid(G)


def test_smoother_tiles_are_tuned_candidates(abi):
    # after a 3-D solve whose finest level is large enough, the tuner has picked
    # a tile for it from its candidate sets; the half sweep is the same for any
    # tile (the cells of one colour are independent), which the V-cycle test on
    # the (96, 64, 64) grid checks against the exact solution
    wl = Workload("tune", (64, 64, 64), (1.0, 1.0, 1.0),
                  bodies=[Body(np.array([0.5, 0.5, 0.5]), sphere_markers(0.2, 120), np.ones(6))], tol=1e-8)
    G = gpu_grid(abi, wl, abi.MIXED)
    try:
        abi.solve_coupled(G, wl.UO(), opts=abi.solve_opts_default())
    finally:
        abi.destroy_grid(G)
    tiles = abi.tuned_smoother_tiles()
    mine = [t for t in tiles if t[:3] == (64, 64, 64) and t[4] == 4]
    assert {t[3] for t in mine} == {1, 3}
    for t in mine:
        assert t[5] in (4, 8) and t[6] in (2, 4, 6, 8, 11, 16, 22, 32)


@pytest.mark.parametrize("dim", [2, 3])
def test_mtilde_couples_bodies_with_minimum_images(abi, dim):
    # several bodies within the single-block limit, coupling requested: one block of all markers,
    # Eq. M_tilde_ij for every pair with minimum-image displacements (one body
    # straddles the periodic seam)
    rng = np.random.default_rng(17)
    if dim == 2:
        n, h = (48, 48), 1.0 / 48
        bodies = [Body(np.array([0.03, 0.5]), disk_markers(0.1, h), rng.standard_normal(3)),
                  Body(np.array([0.55, 0.42]), disk_markers(0.12, h), rng.standard_normal(3))]
    else:
        n, h = (24, 24, 24), 1.0 / 24
        bodies = [Body(np.array([0.97, 0.5, 0.45]), sphere_markers(0.15, 40), rng.standard_normal(6)),
                  Body(np.array([0.45, 0.55, 0.6]), sphere_markers(0.12, 30), rng.standard_normal(6))]
    wl = Workload("coupled", n, (1.0,) * dim, bodies=bodies)
    pr = oracle_problem(wl)
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        o = abi.solve_opts_default()
        o.mob_model = abi.MOB_AUTO | abi.MOB_COUPLED
        abi.prepare(G, o)
        m = pr.N * dim
        out = torch.zeros(m * m, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, out)
        aoh, coef = abi.mobility_defaults(dim)
        if dim == 2:
            ref = mobility.mtilde_2d_steady(pr.q, h, 1.0, 1.0, aoh, list(coef), box=(1.0, 1.0))
        else:
            ref = mobility.mtilde_3d_rpy(pr.q, h, 1.0, 1.0, aoh, periodic=True, box=(1.0, 1.0, 1.0))
        assert rel_err(out.cpu().numpy(), ref) < TOL
    finally:
        abi.destroy_grid(G)
