"""The no-allocation V-cycle entry point against the grid-based one.

ibr_op_vcycle_noalloc exists for callers that cannot call cudaMalloc: an
application whose device memory is all handed to its own pool allocator, a
plug-in running inside a host program that owns the CUDA context, or code that
must not trigger the allocator's device-wide synchronisation.  It keeps its
multigrid coarse levels in a fixed static device array instead.  These tests
call it through the C ABI and compare its result with ibr_op_vcycle (which
uses the grid's own allocations) after each of two consecutive calls, within
the 1e-12 relative tolerance of the other FP64 kernel tests.  The file sorts
last so that a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n,sigma", [((32, 32, 32), 0.0), ((96, 64), 3e3), ((24, 16, 32), 0.0)])
def test_noalloc_vcycle_matches_grid_vcycle_twice(abi, n, sigma):
    d = len(n)
    L = [v / n[0] for v in n]
    kappa = 1.3
    ncell = int(np.prod(n))
    rng = np.random.default_rng(7)
    f = rng.standard_normal(ncell)
    if sigma == 0.0:
        f -= f.mean()
    f_dev = torch.tensor(f, device="cuda")
    u0 = torch.tensor(rng.standard_normal(ncell), device="cuda")
    G = abi.create_grid(d, n, L, precision=abi.FP64)
    try:
        u_ref = u0.clone()
        u_new = u0.clone()
        for call in range(2):
            abi.op_vcycle(G, sigma, kappa, f_dev, u_ref, 1)
            abi.op_vcycle_noalloc(d, n, L, sigma, kappa, f_dev, u_new, 1)
            torch.cuda.synchronize()
            assert _rel(u_new, u_ref) < TOL, (call, _rel(u_new, u_ref))
    finally:
        abi.destroy_grid(G)


def test_noalloc_vcycle_rejects_grids_beyond_the_scratch(abi):
    n = (128, 128, 128)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.IbrError) as e:
        abi.op_vcycle_noalloc(3, n, (1.0, 1.0, 1.0), 0.0, 1.0, f, f, 1)
    assert e.value.code == abi.EINVAL
    assert "static scratch" in abi.last_error()


def test_noalloc_vcycle_rejects_non_cubic_cells(abi):
    # the V-cycle's operator assumes one cell width h on every axis
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(abi.IbrError) as e:
        abi.op_vcycle_noalloc(2, (32, 32), (1.0, 2.0), 0.0, 1.0, f, f, 1)
    assert e.value.code == abi.EINVAL
    assert "cubes" in abi.last_error()
