"""GPU parity of the six-point kernel (IBR_KERNEL_BKP6, the kernel Sec. III.A
uses) against the oracle's, through the C ABI.

The library evaluates the kernel from a closed form of its defining
conditions (elimination in terms of phi(r - 3), one root of the quadratic);
the oracle solves the same conditions by linear algebra.  Spreading and
interpolation agree at rounding level (1e-12), the full constrained solve at
the parity bars of the four-point kernel (1e-9 at residual 1e-10), the 3-D
analytic M~ takes the six-point radius a = 1.47 h (Sec. IV.A), and the
tabulated pair mobility is built with the six-point windows.
"""
import numpy as np
import pytest

from oracle import fft_stokes, ib, mobility
from oracle.system import drag
from synthetic import Body, Workload, disk_markers, sphere_markers

from ._util import flat_fields, gpu_grid, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


def _cases():
    rng = np.random.default_rng(66)
    disk = Workload("bkp6_disk_48x40", (48, 40), (1.2, 1.0), kernel="bkp6", bodies=[
        Body(np.array([0.41, 0.37]), disk_markers(0.14, 1 / 40), rng.standard_normal(3)),
        Body(np.array([0.93, 0.71]), disk_markers(0.09, 1 / 40), rng.standard_normal(3))])
    seam = Workload("bkp6_seam_32", (32, 32), (1.0, 1.0), kernel="bkp6", bodies=[
        Body(np.array([0.02, 0.985]), disk_markers(0.11, 1 / 32), rng.standard_normal(3))])
    sph = Workload("bkp6_sphere_24x20x28", (24, 20, 28), (1.2, 1.0, 1.4), kernel="bkp6", bodies=[
        Body(np.array([0.55, 0.48, 0.71]), sphere_markers(0.22, 60), rng.standard_normal(6))])
    return [disk, seam, sph]


CASES = _cases()
IDS = [c.name for c in CASES]


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_bkp6_spread_interp_parity(abi, wl):
    pr = oracle_problem(wl)
    g = pr.grid
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        abi.prepare(G)
        rng = np.random.default_rng(7)
        lam = rng.standard_normal((pr.N, g.d))
        v = [rng.standard_normal(g.shape) for _ in range(g.d)]
        f_dev = torch.zeros(g.d * g.ncell, dtype=torch.float64, device="cuda")
        abi.op_spread(G, _t(lam), f_dev)
        assert rel_err(f_dev.cpu().numpy(), flat_fields(ib.spread_tilde(g, pr.q, lam))) < 1e-12
        U_dev = torch.zeros(pr.N * g.d, dtype=torch.float64, device="cuda")
        abi.op_interp(G, _t(flat_fields(v)), U_dev)
        assert rel_err(U_dev.cpu().numpy(), ib.interp(g, pr.q, v)) < 1e-12
        y_dev = torch.zeros(pr.size, dtype=torch.float64, device="cuda")
        x = rng.standard_normal(pr.size)
        abi.apply_system(G, _t(x), y_dev)
        assert rel_err(y_dev.cpu().numpy(), pr.matvec(x)) < 1e-12
    finally:
        abi.destroy_grid(G)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_bkp6_solve_matches_oracle(abi, wl, prec):
    pr = oracle_problem(wl)
    vo, po, lo = fft_stokes.solve_coupled(pr, wl.UO())
    G = gpu_grid(abi, wl, getattr(abi, prec))
    try:
        o = abi.solve_opts_default()
        o.tol = 1e-10
        o.max_iters = 400
        info = abi.solve_coupled(G, wl.UO(), opts=o)
        lam, ft = abi.get_forces(G, wl.d)
        n = int(np.prod(wl.n))
        v, p = np.zeros(wl.d * n), np.zeros(n)
        abi.get_fields(G, v, p)
    finally:
        abi.destroy_grid(G)
    assert info.status == abi.OK, info.as_dict()
    for a, b in ((v, flat_fields(vo)), (p, po.ravel()), (lam, lo), (ft, drag(pr, lo))):
        assert rel_err(a, b) < 1e-9, info.as_dict()


def test_bkp6_rpy_radius(abi):
    # 3-D analytic M~ with the six-point radius a = 1.47 h (Sec. IV.A)
    wl = CASES[2]
    pr = oracle_problem(wl)
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        abi.prepare(G)
        dN = pr.N * 3
        out = torch.zeros(dN * dN, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, out)
        M = mobility.mtilde_3d_rpy(wl.bodies[0].rel, pr.grid.h, wl.eta, wl.L[0], 1.47, periodic=True)
        assert rel_err(out.cpu().numpy(), M) < 1e-12
    finally:
        abi.destroy_grid(G)


@pytest.mark.parametrize("idx,bound", [(0, 1.5e-5), (2, 2e-5)], ids=["2d", "3d"])
def test_bkp6_pair_mtilde_matches_oracle(abi, idx, bound):
    # the tabulated pair mobility on a six-point grid; the bound is the FP32
    # arithmetic of the build: 6^d window cells x 2^-24 of the largest entry
    wl = CASES[idx]
    d = wl.d
    G = gpu_grid(abi, wl, abi.MIXED)
    try:
        o = abi.solve_opts_default()
        o.mob_model = abi.MOB_PAIR
        abi.prepare(G, o)
        _, N, _ = abi.sizes(G)
        out = torch.zeros((N * d) ** 2, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, out)
        torch.cuda.synchronize()
        Mg = out.cpu().numpy().reshape(N * d, N * d)
    finally:
        abi.destroy_grid(G)
    pr = oracle_problem(wl)
    Mo = mobility.pair_table_mtilde(pr.grid, pr.q, mobility.pair_sources(wl.n, pr.grid.h, d))
    assert np.array_equal(Mg, Mg.T)
    assert np.abs(Mg - Mo).max() < bound * np.abs(Mo).max()


def test_bkp6_with_walls_rejected(abi):
    with pytest.raises(abi.IbrError) as e:
        abi.create_grid(2, (16, 16), (1.0, 1.0), bc=[abi.PERIODIC, abi.PERIODIC, abi.NOSLIP, abi.NOSLIP],
                        kernel=abi.KERNEL_BKP6)
    assert e.value.code == abi.EINVAL
