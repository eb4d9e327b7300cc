"""Pins for the time-step oracle (advection term and the march).

* A uniform flow has N = 0; discrete momentum is conserved (sum of N_a = 0 in
  a periodic box); for a discretely divergence-free field the centred flux
  form conserves kinetic energy (sum_a v_a . N_a = 0), in a periodic box and
  with no-slip walls.
* Second-order convergence to the analytic (v . grad) v of the Taylor-Green
  vortex u = sin x cos y, v = -cos x sin y: N = (sin 2x, sin 2y) / 2.
* A discrete Poiseuille channel flow (inflow = outflow profile) is a steady
  state of the march: one step leaves it unchanged.
* Any divergence-free field v* is a steady state of the march under the
  body force that balances it, f = -eta Lap v* + rho N(v*): the Euler first
  step and the AB2 steps after it reproduce v* (N != 0 here, so the
  coefficients of the AB2 combination must sum to one).
"""
import numpy as np
import pytest

from oracle import timestep as T
from oracle import walls as W


def _divfree_2d(wg, rng):
    """velocity from a random node stream function: discretely divergence-free"""
    n0, n1 = wg.n
    psi = rng.standard_normal((n1 + 1, n0 + 1))
    if wg.walls[1]:
        psi[0, :] = 0.0
        psi[-1, :] = 0.0
    if wg.walls[0]:
        psi[:, 0] = 0.0
        psi[:, -1] = 0.0
    if not wg.walls[0]:
        psi[:, -1] = psi[:, 0]
    if not wg.walls[1]:
        psi[-1, :] = psi[0, :]
    u = (psi[1:, :-1] - psi[:-1, :-1]) / wg.h   # x-face (i, j): psi(i, j+1) - psi(i, j)
    v = -(psi[:-1, 1:] - psi[:-1, :-1]) / wg.h  # y-face (i, j): -(psi(i+1, j) - psi(i, j))
    return [u, v]


def test_uniform_flow_no_advection():
    wg = W.WallGrid((8, 6), (8 / 6, 1.0), (False, False))
    v = [np.full(wg.shape, 0.7), np.full(wg.shape, -0.3)]
    for Na in T.advect(wg, v):
        assert np.abs(Na).max() < 1e-13


def test_momentum_and_energy_conservation_periodic():
    rng = np.random.default_rng(4)
    wg = W.WallGrid((12, 8), (1.5, 1.0), (False, False))
    v = [rng.standard_normal(wg.shape) for _ in range(2)]
    N = T.advect(wg, v)
    for Na in N:
        assert abs(Na.sum()) < 1e-10 * np.abs(Na).sum()
    vd = _divfree_2d(wg, rng)
    D = wg.D_matrix()
    assert np.abs(D @ np.concatenate([a.ravel() for a in vd])).max() < 1e-10
    Nd = T.advect(wg, vd)
    e = sum(np.sum(vd[a] * Nd[a]) for a in range(2))
    assert abs(e) < 1e-11 * sum(np.sum(np.abs(vd[a] * Nd[a])) for a in range(2))


@pytest.mark.parametrize("walls", [(False, True), (True, True)])
def test_energy_conservation_noslip(walls):
    rng = np.random.default_rng(6)
    wg = W.WallGrid((12, 8), (1.5, 1.0), walls)
    vd = _divfree_2d(wg, rng)
    D = wg.D_matrix()
    assert np.abs(D @ np.concatenate([a.ravel() for a in vd])).max() < 1e-10
    Nd = T.advect(wg, vd)
    e = sum(np.sum(vd[a] * Nd[a]) for a in range(2))
    assert abs(e) < 1e-11 * sum(np.sum(np.abs(vd[a] * Nd[a])) for a in range(2))


def test_taylor_green_second_order():
    errs = []
    for n in (16, 32, 64):
        L = 2 * np.pi
        wg = W.WallGrid((n, n), (L, L), (False, False))
        h = wg.h
        xf = np.arange(n) * h           # face coordinate along its own axis
        xc = (np.arange(n) + 0.5) * h   # cell centres
        u = np.sin(xf)[None, :] * np.cos(xc)[:, None]
        v = -np.cos(xc)[None, :] * np.sin(xf)[:, None]
        N = T.advect(wg, [u, v])
        ex = 0.5 * np.sin(2 * xf)[None, :] * np.ones((n, 1))
        ey = 0.5 * np.sin(2 * xf)[:, None] * np.ones((1, n))
        errs.append(max(np.abs(N[0] - ex).max(), np.abs(N[1] - ey).max()))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9), (errs, rates)


def test_poiseuille_is_a_steady_state_of_the_march():
    eta, rho, dt = 0.05, 1.0, 0.02
    wg = W.WallGrid((12, 8), (1.5, 1.0), (True, True), eta=eta, rho=rho, dt=dt)
    ny = 8
    Tm = W._lap1d(ny, "cdir").toarray()
    ud = np.linalg.solve(-(eta / wg.h ** 2) * Tm, np.ones(ny))
    bd = wg.zero_data()
    bd[(0, 0)][0][:] = ud
    bd[(0, 1)][0][:] = ud
    prob = W.WallProblem(wg, np.zeros((0, 2)))
    v0 = [np.broadcast_to(ud[:, None], wg.shape).copy(), np.zeros(wg.shape)]
    N0 = T.advect(wg, v0, bd)
    assert max(np.abs(Na).max() for Na in N0) < 1e-12 * np.abs(ud).max() ** 2 / wg.h
    states, changes = T.march(prob, np.zeros(0), bd, v0, 2)
    assert max(changes) < 1e-12
    v1, _, _ = prob.split(states[-1])
    assert np.abs(v1[0] - v0[0]).max() < 1e-11 * np.abs(ud).max()


@pytest.mark.parametrize("walls", [(False, False), (False, True)])
def test_forced_steady_state_with_advection(walls):
    rng = np.random.default_rng(12)
    eta, rho, dt = 0.3, 2.0, 0.01
    wg = W.WallGrid((12, 8), (1.5, 1.0), walls, eta=eta, rho=rho, dt=dt)
    vs = _divfree_2d(wg, rng)
    bd = wg.zero_data()
    N = T.advect(wg, vs, bd)
    assert max(np.abs(Na).max() for Na in N) > 1.0
    steady = W.WallGrid(wg.n, wg.L, walls, eta=eta)
    Av = (steady.A_matrix() @ np.concatenate([a.ravel() for a in vs])).reshape(2, *wg.shape)
    f = [Av[c] + rho * N[c] for c in range(2)]
    prob = W.WallProblem(wg, np.zeros((0, 2)))
    states, changes = T.march(prob, np.zeros(0), bd, vs, 3, force=f)
    assert max(changes) < 1e-11, changes
