"""GPU parity of the time-stepped path (Sec. VII.F): the advection term and
ibr_advance (backward Euler + AB2 with the constrained solve each step)
against the oracle's march, through the C ABI.

Tolerances: N(v) is a fixed FP64 stencil (1e-12 relative); each step's solve
goes to a relative residual of 1e-11 and the states after a few steps agree
to 1e-8 (the per-step solve error is not amplified by the stable backward-
Euler step, but it accumulates over steps).
"""
import numpy as np
import pytest

from oracle import timestep as T
from oracle import walls as W
from oracle.ib import apply_K
from synthetic import Body, Workload, disk_markers, nozzle, parabolic_inflow

from ._util import gpu_grid, oracle_wall_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


def _inflow_case(n=(48, 16), rho=1.0, dt=0.02, eta=0.05, walls=(True, True), seed=2):
    rng = np.random.default_rng(seed)
    h = 1.0 / n[1]
    L = (n[0] * h, 1.0)
    bodies = [Body(np.array([0.45 * L[0], 0.45]), disk_markers(3.0 * h, h), np.zeros(3))]
    wl = Workload(f"step_{n[0]}x{n[1]}", n, L, eta=eta, rho=rho, dt=dt, bodies=bodies, tol=1e-11, walls=walls)
    data = None
    if walls[0]:
        data = {}
        for s in (0, 1):
            v = np.zeros((2, n[1]))
            v[0] = parabolic_inflow(n[1], U=1.0)
            data[(0, s)] = v
    return wl, data


def _bd(prob, data):
    bd = prob.g.zero_data()
    for k, v in (data or {}).items():
        bd[k] = np.asarray(v, dtype=np.float64).reshape(bd[k].shape)
    return bd


@pytest.mark.parametrize("walls", [(True, True), (False, True), (False, False)])
def test_advect_matches_oracle(abi, walls):
    wl, data = _inflow_case(walls=walls)
    prob, _, _ = oracle_wall_problem(wl)
    wg = prob.g
    rng = np.random.default_rng(1)
    v = [rng.standard_normal(wg.shape) for _ in range(2)]
    N = T.advect(wg, v, _bd(prob, data))
    G = gpu_grid(abi, wl, abi.FP64, data=data)
    try:
        vt = torch.tensor(np.concatenate([a.ravel() for a in v]), device="cuda")
        Nt = torch.zeros_like(vt)
        abi.op_advect(G, vt, Nt)
        Ng = Nt.cpu().numpy()
    finally:
        abi.destroy_grid(G)
    ref = np.concatenate([a.ravel() for a in N])
    assert np.abs(Ng - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
@pytest.mark.parametrize("walls", [(True, True), (False, True)])
def test_march_matches_oracle(abi, prec, walls):
    wl, data = _inflow_case(walls=walls)
    prob, rel, body = oracle_wall_problem(wl)
    bd = _bd(prob, data)
    Wv = -apply_K(rel, body, wl.UO(), 2).ravel()
    v0 = [np.zeros(prob.g.shape), np.zeros(prob.g.shape)]
    force = None
    if not walls[0]:  # a channel driven by a body force
        force = [np.full(prob.g.shape, 1.0), np.zeros(prob.g.shape)]
    states, changes = T.march(prob, Wv, bd, v0, 4, force=force)
    G = gpu_grid(abi, wl, getattr(abi, prec), data=data)
    try:
        o = abi.solve_opts_default()
        o.tol = 1e-11
        o.max_iters = 400
        fg = None if force is None else np.concatenate([a.ravel() for a in force])
        info = abi.advance(G, wl.UO(), 4, g=fg, opts=o)
        assert info.status == abi.OK, info.as_dict()
        assert info.steps == 4
        n = int(np.prod(wl.n))
        v = np.zeros(2 * n)
        p = np.zeros(n)
        abi.get_fields(G, v, p)
        lam, _ = abi.get_forces(G, 2)
    finally:
        abi.destroy_grid(G)
    vo, po, lo = prob.split(states[-1])
    assert rel_err(v, np.concatenate([a.ravel() for a in vo])) < 1e-8, info.as_dict()
    assert rel_err(p, po) < 1e-8
    assert rel_err(lam, lo) < 1e-8
    assert abs(info.change - changes[-1]) <= 1e-6 * changes[-1]


def test_step_from_a_given_state(abi):
    """ibr_set_velocity + a body force: one step from a divergence-free field
    with advection (N != 0) matches the oracle's step from the same state"""
    wl, _ = _inflow_case(walls=(False, True))
    prob, rel, body = oracle_wall_problem(wl)
    wg = prob.g
    rng = np.random.default_rng(3)
    n0, n1 = wg.n
    psi = rng.standard_normal((n1 + 1, n0 + 1))
    psi[0, :] = psi[-1, :] = 0.0
    psi[:, -1] = psi[:, 0]
    vs = [(psi[1:, :-1] - psi[:-1, :-1]) / wg.h, -(psi[:-1, 1:] - psi[:-1, :-1]) / wg.h]
    f = [np.full(wg.shape, 0.5), np.zeros(wg.shape)]
    Wv = -apply_K(rel, body, wl.UO(), 2).ravel()
    states, changes = T.march(prob, Wv, _bd(prob, None), vs, 2, force=f)
    G = gpu_grid(abi, wl, abi.FP64)
    try:
        o = abi.solve_opts_default()
        o.tol = 1e-11
        abi.set_velocity(G, np.concatenate([a.ravel() for a in vs]))
        info = abi.advance(G, wl.UO(), 2, g=np.concatenate([a.ravel() for a in f]), opts=o)
        assert info.status == abi.OK, info.as_dict()
        n = int(np.prod(wl.n))
        v = np.zeros(2 * n)
        abi.get_fields(G, v, None)
    finally:
        abi.destroy_grid(G)
    vo, _, _ = prob.split(states[-1])
    assert rel_err(v, np.concatenate([a.ravel() for a in vo])) < 1e-8
    assert abs(info.change - changes[-1]) <= 1e-6 * changes[-1]


def test_steady_state_stops_the_march(abi):
    """a channel with the discrete Poiseuille profile at inflow and outflow
    and a fixed disk: from rest the march reaches a steady state (change per
    step below 1e-6) and stops there by itself"""
    eta = 0.05
    wl, _ = _inflow_case(eta=eta)
    wl.bodies = [Body(np.array([0.5 * wl.L[0], 0.5]), disk_markers(3.0 / 16, 1 / 16), np.zeros(3))]
    ny = wl.n[1]
    h = 1.0 / ny
    Tm = W._lap1d(ny, "cdir").toarray()
    ud = np.linalg.solve(-(eta / h ** 2) * Tm, np.ones(ny))
    data = {}
    for s in (0, 1):
        v = np.zeros((2, ny))
        v[0] = ud
        data[(0, s)] = v
    G = gpu_grid(abi, wl, abi.MIXED, data=data)
    try:
        o = abi.solve_opts_default()
        o.tol = 1e-10
        info0 = abi.advance(G, wl.UO(), 200, steady_tol=1e-6, opts=o)
        assert info0.status == abi.OK and info0.steps < 200, info0.as_dict()
        assert info0.change <= 1e-6
    finally:
        abi.destroy_grid(G)


def test_nozzle_march_with_true_mobility(abi):
    """The nozzle at Re = 10 on a 128 x 64 grid: three steps from rest with
    the precomputed true mobility, mixed precision, per-step tolerance 1e-8;
    the state follows the oracle's march to 1e-6."""
    wl = nozzle(n=(128, 64), Re=10.0)
    data = {}
    for s in (0, 1):
        v = np.zeros((2, wl.n[1]))
        v[0] = parabolic_inflow(wl.n[1])
        data[(0, s)] = v
    prob, rel, body = oracle_wall_problem(wl)
    states, changes = T.march(prob, np.zeros(prob.N * 2), _bd(prob, data), [np.zeros(prob.g.shape)] * 2, 3)
    G = gpu_grid(abi, wl, abi.MIXED, data=data)
    try:
        o = abi.solve_opts_default()
        o.tol = 1e-8
        o.mob_model = abi.MOB_TRUE
        info = abi.advance(G, wl.UO(), 3, opts=o)
        assert info.status == abi.OK, info.as_dict()
        assert info.iters_total <= 3 * 40, info.as_dict()
        n = int(np.prod(wl.n))
        v = np.zeros(2 * n)
        abi.get_fields(G, v, None)
    finally:
        abi.destroy_grid(G)
    vo, _, _ = prob.split(states[-1])
    assert rel_err(v, np.concatenate([a.ravel() for a in vo])) < 1e-6
