"""Pins for the oracle's kernel and MAC operators (CPU only).

Each check is fixed by the mathematics, not by re-typing the oracle:
kernel moment conditions by brute force, closed-form kernel values, the
assembled-vs-matrix-free operators, D = -G^T, and the periodic Laplacian
spectrum in closed form.
"""
import json
import os

import numpy as np
import pytest

from oracle.mac import Grid, flat, unflat
from oracle.peskin import phi, support_weights

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_peskin_closed_form_values():
    pts = json.load(open(os.path.join(GOLD, "peskin4_values.json")))["points"]
    for p in pts:
        assert phi(np.array([p["r"]]))[0] == pytest.approx(p["phi"], abs=1e-15)
        assert phi(np.array([-p["r"]]))[0] == pytest.approx(p["phi"], abs=1e-15)


def test_peskin_moment_conditions_bruteforce():
    # 10^4 shifts; sums over all integer nodes in a wide window
    s = np.linspace(-3.0, 3.0, 10001)
    j = np.arange(-8, 9)
    r = s[:, None] - j[None, :]
    w = phi(r)
    assert np.max(np.abs(w.sum(1) - 1.0)) < 1e-14
    assert np.max(np.abs((r * w).sum(1))) < 1e-14
    even = (j % 2 == 0)
    assert np.max(np.abs(w[:, even].sum(1) - 0.5)) < 1e-14
    assert np.max(np.abs((w * w).sum(1) - 3.0 / 8.0)) < 1e-14
    assert np.all(w >= 0)


def test_peskin_support_window_matches_full_sum():
    rng = np.random.default_rng(0)
    s = rng.uniform(-10, 10, 500)
    j0, w = support_weights(s)
    assert np.allclose(w.sum(1), 1.0, atol=1e-14)
    # every node outside the window has zero weight
    for k in (-1, 4):
        assert np.all(phi(s - (j0 + k)) == 0.0)


@pytest.mark.parametrize("n", [(6, 5), (4, 3, 5)])
def test_div_is_minus_grad_transpose_and_matches_matrix_free(n):
    g = Grid(n, [v / n[0] for v in n])
    rng = np.random.default_rng(1)
    G = g.G_matrix()
    p = rng.standard_normal(g.shape)
    v = [rng.standard_normal(g.shape) for _ in range(g.d)]
    assert np.allclose(G @ p.ravel(), flat(g.grad(p)), atol=1e-12)
    # D = -G^T: compare the matrix-free divergence with -G^T v
    assert np.allclose(-(G.T @ flat(v)), g.div(v).ravel(), atol=1e-12)
    Lm = g.lap_matrix()
    assert np.allclose(Lm @ p.ravel(), g.lap(p).ravel(), atol=1e-12)
    # D G = h^-2 Lap on cell-centred scalars (the pressure Poisson operator L_p = h^2 D G)
    assert np.allclose(g.div(g.grad(p)), g.lap(p) / g.h ** 2, atol=1e-9)


@pytest.mark.parametrize("n", [(6, 6), (4, 4, 4)])
def test_periodic_laplacian_spectrum_closed_form(n):
    g = Grid(n)
    ev = np.sort(np.linalg.eigvalsh(g.lap_matrix().toarray()))
    ks = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    lam = -sum(4.0 * np.sin(np.pi * k / m) ** 2 for k, m in zip(ks, n))
    assert np.allclose(ev, np.sort(lam.ravel()), atol=1e-12)


def test_viscous_operator_scaling():
    # A = eta h^-2 (beta^-1 I - Lap) with beta = (eta/rho) dt / h^2 (Eq. A_def)
    g = Grid((8, 8), eta=2.0, rho=3.0, dt=0.01)
    rng = np.random.default_rng(2)
    v = [rng.standard_normal(g.shape) for _ in range(2)]
    beta = (g.eta / g.rho) * g.dt / g.h ** 2
    Av = g.apply_A(v)
    for a in range(2):
        ref = g.eta / g.h ** 2 * (v[a] / beta - g.lap(v[a]))
        assert np.allclose(Av[a], ref, rtol=1e-12, atol=1e-9)


def test_flat_roundtrip():
    g = Grid((4, 3, 2), (1.0, 0.75, 0.5))
    rng = np.random.default_rng(3)
    v = [rng.standard_normal(g.shape) for _ in range(3)]
    w = unflat(g, flat(v), 3)
    for a in range(3):
        assert np.array_equal(v[a], w[a])
