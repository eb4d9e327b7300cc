"""Pins for the wall-bounded oracle (App. D).

* Route K (Kronecker-assembled sparse operators) equals route X (the ghost
  extension u_ext = E u + c applied literally) on random fields and random
  wall data; D = -G^T; A symmetric.
* The composed interpolation J_0 E equals a brute-force kernel sum over a
  two-layer ghost-extended grid; markers on a no-slip wall interpolate
  exactly zero (App. D: the extension makes the interpolated velocity vanish
  at a no-slip boundary).
* Exact discrete solutions: plane Couette flow (linear profile, exact for the
  linear-extrapolation ghost rule) and pressure-driven channel flow whose
  inflow/outflow profile is the discrete 1-D Poiseuille profile.
* The sparse LU solve equals an independent route: exact velocity solves by
  separable DST/DFT transforms with a dense pressure Schur complement, and,
  with markers, the Schur route M = J L^-1 S of Sec. V.A.
"""
import numpy as np
import pytest

from oracle import walls as W

CASES = [
    ("2d_box", (8, 6), (8 / 6, 1.0), (True, True)),
    ("2d_channel", (8, 6), (8 / 6, 1.0), (False, True)),
    ("3d_duct", (4, 6, 4), (4 / 6, 1.0, 4 / 6), (False, True, True)),
]


def _rand_data(wg, rng):
    return {k: rng.standard_normal(v.shape) for k, v in wg.zero_data().items()}


@pytest.mark.parametrize("name,n,L,walls", CASES)
@pytest.mark.parametrize("rho", [0.0, 2.0])
def test_route_k_equals_route_x(name, n, L, walls, rho):
    rng = np.random.default_rng(11)
    wg = W.WallGrid(n, L, walls, eta=0.7, rho=rho, dt=0.05)
    d, nc = wg.d, wg.ncell
    v = [rng.standard_normal(wg.shape) for _ in range(d)]
    p = rng.standard_normal(wg.shape)
    bd = _rand_data(wg, rng)
    mom, div = wg.apply_full(v, p, bd)
    mom0, div0 = wg.apply_full([0 * x for x in v], 0 * p, bd)
    x = np.concatenate([np.concatenate([a.ravel() for a in v])])
    Av = wg.A_matrix() @ x
    Gp = wg.G_matrix() @ p.ravel()
    for c in range(d):
        lin = (Av + Gp)[c * nc:(c + 1) * nc].reshape(wg.shape)
        bm = wg.boundary_mask(c)
        assert np.allclose(lin[~bm], (mom[c] - mom0[c])[~bm], rtol=1e-12, atol=1e-9)
        assert np.array_equal(lin[bm], v[c][bm])
        assert np.array_equal(mom[c][bm], v[c][bm])
    assert np.allclose((wg.D_matrix() @ x).reshape(wg.shape), div - div0, rtol=1e-12, atol=1e-9)


def test_boundary_data_terms_closed_form():
    """The data terms of single entries, from the ghost rules by hand."""
    wg = W.WallGrid((6, 4), (1.5, 1.0), (True, True), eta=1.3)
    bd = wg.zero_data()
    bd[(0, 0)][0][2] = 5.0  # normal velocity on x = 0 at cell row j = 2
    bd[(1, 1)][0][3] = 7.0  # tangential x-velocity on y = L at face column i = 3
    z = np.zeros(wg.shape)
    mom0, div0 = wg.apply_full([z, z], z, bd)
    k = wg.eta / wg.h ** 2
    # face i = 1 sees the wall face i = 0 as its x-neighbour
    assert np.isclose(mom0[0][2, 1], -k * 5.0)
    # cell-centred row next to the top wall: ghost = 2 u_w - u
    assert np.isclose(mom0[0][3, 3], -2 * k * 7.0)
    # the divergence of cell (0, 2) loses the inflow through its low face
    assert np.isclose(div0[2, 0], -5.0 / wg.h)
    assert np.count_nonzero(mom0[0]) == 2 and np.count_nonzero(div0) == 1


@pytest.mark.parametrize("name,n,L,walls", CASES)
def test_operator_structure(name, n, L, walls):
    wg = W.WallGrid(n, L, walls, eta=1.0, rho=1.0, dt=0.1)
    A = wg.A_matrix()
    assert abs(A - A.T).max() == 0.0
    G = wg.G_matrix()
    assert abs(wg.D_matrix() + G.T).max() == 0.0
    # no gradient on wall faces; the pressure constant is the only null vector of G
    bm = np.concatenate([wg.boundary_mask(c).ravel() for c in range(wg.d)])
    assert abs(G[bm]).max() == 0.0 if bm.any() else True
    assert np.abs(G @ np.ones(wg.ncell)).max() < 1e-12


def _near_wall_markers(wg, rng, m):
    q = rng.uniform(0, 1, (m, wg.d)) * np.array(wg.L)
    # push some markers into the kernel support of walls and corners
    for i in range(m):
        for a in range(wg.d):
            if wg.walls[a] and i % 2 == 0:
                q[i, a] = rng.uniform(0, 2.5) * wg.h if i % 4 == 0 else wg.L[a] - rng.uniform(0, 2.5) * wg.h
    return q


@pytest.mark.parametrize("name,n,L,walls", CASES)
def test_interp_equals_bruteforce_extension(name, n, L, walls):
    rng = np.random.default_rng(5)
    wg = W.WallGrid(n, L, walls)
    q = _near_wall_markers(wg, rng, 9)
    v = [rng.standard_normal(wg.shape) for _ in range(wg.d)]
    Jm = wg.J_matrix(q)
    x = np.concatenate([a.ravel() for a in v])
    got = (Jm @ x).reshape(-1, wg.d)
    ref = wg.interp_bruteforce(v, q)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-13)
    # wall faces carry data, not unknowns: no weight on them
    bm = np.concatenate([wg.boundary_mask(c).ravel() for c in range(wg.d)])
    assert np.abs(Jm[:, bm]).max() == 0.0 if bm.any() else True


@pytest.mark.parametrize("name,n,L,walls", CASES)
def test_interp_vanishes_on_noslip_wall(name, n, L, walls):
    rng = np.random.default_rng(8)
    wg = W.WallGrid(n, L, walls)
    v = [rng.standard_normal(wg.shape) for _ in range(wg.d)]
    x = np.concatenate([a.ravel() for a in v])
    for a in range(wg.d):
        if not wg.walls[a]:
            continue
        q = rng.uniform(0.2, 0.8, (4, wg.d)) * np.array(wg.L)
        q[:2, a] = 0.0
        q[2:, a] = wg.L[a]
        out = wg.J_matrix(q) @ x
        assert np.abs(out).max() < 1e-13


@pytest.mark.parametrize("rho", [0.0, 3.0])
@pytest.mark.parametrize("U0,U1", [(0.0, 1.3), (-0.6, 0.0), (0.4, 1.1)])
def test_couette_exact(rho, U0, U1):
    """Walls at y = 0 and y = 1 sliding at U0 and U1: v_x = U0 + (U1 - U0) y,
    v_y = 0, pi = 0."""
    wg = W.WallGrid((8, 8), (1.0, 1.0), (False, True), eta=0.8, rho=rho, dt=0.1)
    bd = wg.zero_data()
    bd[(1, 0)][0][:] = U0
    bd[(1, 1)][0][:] = U1
    y = (np.arange(8) + 0.5) * wg.h
    ux = np.broadcast_to((U0 + (U1 - U0) * y)[:, None], wg.shape).copy()
    g = [wg.sigma * ux, np.zeros(wg.shape)]  # steady profile of the unsteady operator
    prob = W.WallProblem(wg, np.zeros((0, 2)))
    b = prob.rhs(np.zeros(0), g_force=g, bd=bd)
    x = prob.solve(b)
    v, p, _ = prob.split(x)
    assert np.abs(v[0] - ux).max() < 1e-12
    assert np.abs(v[1]).max() < 1e-12
    assert np.abs(p).max() < 1e-10


def test_poiseuille_exact():
    """Channel [0, 1.5] x [0, 1], inflow = outflow = the discrete 1-D
    Poiseuille profile for a unit pressure gradient: the flow is that profile
    everywhere, v_y = 0, pi linear in x."""
    eta = 0.9
    wg = W.WallGrid((12, 8), (1.5, 1.0), (True, True), eta=eta)
    h = wg.h
    ny = 8
    T = W._lap1d(ny, "cdir").toarray()
    ud = np.linalg.solve(-(eta / h ** 2) * T, np.ones(ny))  # -eta u'' = -dp/dx = 1
    bd = wg.zero_data()
    bd[(0, 0)][0][:] = ud
    bd[(0, 1)][0][:] = ud
    prob = W.WallProblem(wg, np.zeros((0, 2)))
    b = prob.rhs(np.zeros(0), bd=bd)
    x = prob.solve(b)
    v, p, _ = prob.split(x)
    assert np.abs(v[0] - ud[:, None]).max() < 1e-11 * np.abs(ud).max()
    assert np.abs(v[1]).max() < 1e-11 * np.abs(ud).max()
    xc = (np.arange(12) + 0.5) * h
    pe = -(xc - xc.mean())
    assert np.abs(p - pe[None, :]).max() < 1e-10


@pytest.mark.parametrize("name,n,L,walls", CASES)
@pytest.mark.parametrize("rho", [0.0, 2.0])
def test_sparse_lu_equals_dst_route(name, n, L, walls, rho):
    rng = np.random.default_rng(21)
    wg = W.WallGrid(n, L, walls, eta=1.1, rho=rho, dt=0.05)
    d = wg.d
    bd = _rand_data(wg, rng)
    # no net flux through the walls (solvability of -D v = h)
    for a in range(d):
        if wg.walls[a]:
            lo, hi = bd[(a, 0)][a], bd[(a, 1)][a]
            hi += lo.mean() - hi.mean()
    g = [rng.standard_normal(wg.shape) for _ in range(d)]
    prob = W.WallProblem(wg, np.zeros((0, d)))
    b = prob.rhs(np.zeros(0), g_force=g, bd=bd)
    x = prob.solve(b)
    assert prob.residual(x, b) < 1e-12
    nc = wg.ncell
    gb = [b[c * nc:(c + 1) * nc].reshape(wg.shape) for c in range(d)]
    hb = b[d * nc:(d + 1) * nc].reshape(wg.shape)
    v2, p2 = W.stokes_solve_dst(wg, gb, hb)
    v, p, _ = prob.split(x)
    for c in range(d):
        assert np.allclose(v[c], v2[c], rtol=1e-10, atol=1e-10 * np.abs(v[c]).max())
    assert np.allclose(p, p2, rtol=1e-10, atol=1e-10 * np.abs(p).max())


@pytest.mark.parametrize("name,n,L,walls", CASES[:2] + [CASES[2]])
def test_constrained_solve_with_markers(name, n, L, walls):
    rng = np.random.default_rng(4)
    wg = W.WallGrid(n, L, walls, eta=1.0, rho=1.0 if name == "2d_box" else 0.0, dt=0.1)
    d = wg.d
    q = _near_wall_markers(wg, rng, 4)
    prob = W.WallProblem(wg, q)
    Wv = rng.standard_normal(prob.N * d)
    b = prob.rhs(Wv)
    x = prob.solve(b)
    assert prob.residual(x, b) < 1e-11
    v, p, lam = prob.split(x)
    xv = np.concatenate([a.ravel() for a in v])
    # constraints: -J v = W, divergence free
    assert np.allclose(-prob.J @ xv, Wv, atol=1e-10 * np.abs(Wv).max())
    assert np.abs(wg.D_matrix() @ xv).max() < 1e-9 * np.abs(xv).max() / wg.h
    x2 = W.solve_schur_dst(prob, b)
    assert np.linalg.norm(x - x2) / np.linalg.norm(x) < 1e-9
