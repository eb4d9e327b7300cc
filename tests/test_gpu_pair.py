"""IBR_MOB_PAIR on the GPU: the approximate mobility from the grid's own
tabulated pair mobility (periodic grids).

  - the dense M~ block the library builds equals the oracle's
    pair_table_mtilde (same source points) to the precision of its FP32
    arithmetic: an FP32 table, FP32 kernel weights and FP32 sums over the
    4^d window cells (each sum's rounding is at most 4^d * 2^-24 ~ 4e-6 of
    the largest table value, typically far less): 5e-6 of the largest entry,
    one block coupling all bodies;
  - the constrained solve with it matches the oracle (1e-9 at residual
    1e-10): M~ changes iteration counts only (Sec. V.A);
  - it needs fewer outer iterations than the analytic forms on multi-body
    problems.
"""
import numpy as np
import pytest

from oracle import fft_stokes, mobility
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


def _two_disks(n=32):
    rng = np.random.default_rng(8)
    h = 1.0 / n
    return Workload(f"pair_two_disks_{n}", (n, n), (1.0, 1.0), bodies=[
        Body(np.array([0.31, 0.52]), disk_markers(0.12, h), rng.standard_normal(3)),
        Body(np.array([0.66, 0.47]), disk_markers(0.1, h), rng.standard_normal(3))], tol=1e-10)


def _sphere(n=16):
    rng = np.random.default_rng(9)
    h = 1.0 / n
    return Workload(f"pair_sphere_{n}", (n, n, n), (1.0, 1.0, 1.0), bodies=[
        Body(np.array([0.47, 0.52, 0.55]), sphere_markers(3.2 * h, 40), rng.standard_normal(6))], tol=1e-10)


def _opts(abi, **kw):
    o = abi.solve_opts_default()
    o.tol = 1e-10
    o.max_iters = 400
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("mk", [_two_disks, _sphere], ids=["2d_two_disks", "3d_sphere"])
def test_pair_mtilde_matches_oracle(abi, mk):
    wl = mk()
    d = wl.d
    G = gpu_grid(abi, wl, abi.MIXED)
    try:
        abi.prepare(G, _opts(abi, mob_model=abi.MOB_PAIR))
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
    assert np.abs(Mg - Mo).max() < 5e-6 * np.abs(Mo).max()


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
@pytest.mark.parametrize("mk", [_two_disks, _sphere], ids=["2d_two_disks", "3d_sphere"])
def test_pair_solve_matches_oracle(abi, mk, prec):
    wl = mk()
    G = gpu_grid(abi, wl, getattr(abi, prec))
    try:
        info = abi.solve_coupled(G, wl.UO(), opts=_opts(abi, mob_model=abi.MOB_PAIR))
        lam, ft = abi.get_forces(G, wl.d)
        nc = int(np.prod(wl.n))
        v, p = np.zeros(wl.d * nc), np.zeros(nc)
        abi.get_fields(G, v, p)
    finally:
        abi.destroy_grid(G)
    assert info.status == abi.OK
    pr = oracle_problem(wl)
    vo, po, lo = fft_stokes.solve_coupled(pr, wl.UO())
    assert rel_err(v, flat_fields(vo)) < 1e-9 and rel_err(p, po) < 1e-9
    assert rel_err(lam, lo) < 1e-9 and rel_err(ft, drag(pr, lo)) < 1e-9


def test_pair_needs_fewer_iterations(abi):
    wl = _two_disks(64)
    its = {}
    for name, model in (("auto", abi.MOB_AUTO), ("pair", abi.MOB_PAIR)):
        G = gpu_grid(abi, wl, abi.MIXED)
        try:
            its[name] = abi.solve_coupled(G, wl.UO(), opts=_opts(abi, mob_model=model, tol=1e-8)).iters
        finally:
            abi.destroy_grid(G)
    assert its["pair"] < its["auto"], its


def test_pair_rejects_walls(abi):
    G = abi.create_grid(2, (16, 16), (1.0, 1.0), bc=[abi.PERIODIC, abi.PERIODIC, abi.NOSLIP, abi.NOSLIP])
    try:
        b = abi.add_body(G, (0.5, 0.5))
        abi.set_markers(G, b, disk_markers(0.15, 1 / 16))
        with pytest.raises(abi.IbrError) as e:
            abi.prepare(G, _opts(abi, mob_model=abi.MOB_PAIR))
        assert e.value.code == abi.EINVAL
    finally:
        abi.destroy_grid(G)
