"""Pins for the oracle's six-point kernel (Bao, Kaye and Peskin; the kernel
Sec. III.A uses) and for the J, S built on it (CPU).

* its defining conditions, checked by brute force over many shifts: sums of
  phi, of the even and odd nodes, the first three moments and the sum of
  squares (the oracle solves for the weights; these sums re-evaluate phi);
* three continuous derivatives: the third divided difference has no jump at
  the integers (the property the constant K is chosen for), the fourth does;
* symmetry and support [-3, 3];
* the marker's effective hydrodynamic radius: the paper quotes a = 1.47 h for
  the six-point kernel and a = 1.25 h for the four-point kernel (Sec. IV.A);
  the oracle's self-mobility of one marker in a periodic box, averaged over
  positions and corrected for the periodic images with Eq. drag_periodic,
  reproduces both;
* J = h^d S^T (adjointness) and partition of unity with the wider window.
"""
import json
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import bkp6, fft_stokes, ib, peskin
from oracle.mac import Grid, flat
from oracle.system import Problem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_defining_conditions_by_brute_force():
    rng = np.random.default_rng(3)
    j = np.arange(-12, 13)
    for s in np.concatenate([rng.uniform(-6, 6, 200), [0.0, 0.5, 1.0, -2.0, 2.5]]):
        x = s - j
        p = bkp6.phi(x)
        assert abs(p.sum() - 1.0) < 1e-13
        assert abs(p[j % 2 == 0].sum() - 0.5) < 1e-13
        assert abs((x * p).sum()) < 1e-13
        assert abs((x * x * p).sum() - bkp6.K) < 1e-13
        assert abs((x ** 3 * p).sum()) < 1e-12
        assert abs((p * p).sum() - bkp6.C) < 1e-13
    assert bkp6.K == pytest.approx(59.0 / 60.0 - np.sqrt(29.0) / 20.0, rel=1e-15)


def test_three_continuous_derivatives():
    # third divided differences just left and right of each integer: for a
    # C^3 function they differ by about |phi^(4)| x 5 steps (< 0.01 here); a
    # K off by 0.006 already leaves jumps of 0.02-0.08 (checked when this
    # pin was written), the fourth difference jumps by O(1)
    hstep = 1e-4
    x = np.arange(-3.2, 3.2 + hstep / 2, hstep)
    f = bkp6.phi(x)
    d3 = np.diff(f, 3) / hstep ** 3
    d4 = np.diff(f, 4) / hstep ** 4
    for k in (-3, -2, -1, 0, 1, 2, 3):
        i = int(round((k + 3.2) / hstep))
        assert abs(d3[i + 1] - d3[i - 4]) < 0.01, (k, d3[i - 4], d3[i + 1])
    i = int(round((1 + 3.2) / hstep))
    assert abs(d4[i + 2] - d4[i - 6]) > 1.0


def test_symmetry_and_support():
    x = np.linspace(-4, 4, 801)
    f = bkp6.phi(x)
    assert np.allclose(f, bkp6.phi(-x), atol=1e-15)
    assert np.all(f[np.abs(x) >= 3.0] == 0.0)
    assert f.max() == pytest.approx(bkp6.phi(np.array([0.0]))[0])
    j0, w = bkp6.support_weights(np.array([7.3]))
    assert j0[0] == 5 and np.allclose(w[0], bkp6.phi(7.3 - np.arange(5, 11)), atol=1e-15)


def _hydrodynamic_radius(kernel, n=32, positions=6):
    """a/h from the self-mobility of one marker in a periodic box of n^3
    cells (unit box, eta = 1), averaged over positions, inverted through the
    periodic drag of a sphere (Eq. drag_periodic, Sec. VII.C)"""
    c = json.load(open(os.path.join(GOLD, "paper_constants.json")))["drag_periodic_3d_coefficients"]["value"]
    g = Grid((n, n, n), kernel=kernel)
    rng = np.random.default_rng(11)
    mus = []
    for _ in range(positions):
        q = rng.uniform(0.3, 0.7, (1, 3))
        pr = Problem(g, q, np.zeros((1, 3)), np.array([0]), 1)
        mus.append(np.trace(fft_stokes.mobility_true(pr)) / 3.0)
    mu = float(np.mean(mus))

    def drag(R):
        return 6 * np.pi * R / (1 - c[0] * R + c[1] * R ** 3 + c[2] * R ** 6)

    return brentq(lambda R: drag(R) - 1.0 / mu, 1e-3, 0.3) * n


@pytest.mark.parametrize("kernel,paper", [("bkp6", 1.47), ("peskin4", 1.25)])
def test_hydrodynamic_radius_matches_paper(kernel, paper):
    a = _hydrodynamic_radius(kernel)
    assert abs(a - paper) < 0.03, a


@pytest.mark.parametrize("n", [(12, 12), (8, 9, 10)])
def test_six_point_J_S_adjoint_and_partition_of_unity(n):
    g = Grid(n, [v / n[0] for v in n], kernel="bkp6")
    rng = np.random.default_rng(4)
    q = rng.uniform(0, 1, (5, g.d)) * np.array(g.L)
    v = [rng.standard_normal(g.shape) for _ in range(g.d)]
    lam = rng.standard_normal((5, g.d))
    lhs = np.sum(ib.interp(g, q, v) * lam)
    rhs = g.h ** g.d * np.dot(flat(v), flat(ib.spread(g, q, lam)))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    assert np.allclose(ib.interp(g, q, v), ib.interp_bruteforce(g, q, v), atol=1e-13)
    const = [np.full(g.shape, 2.0 + a) for a in range(g.d)]
    assert np.allclose(ib.interp(g, q, const), [[2.0 + a for a in range(g.d)]] * 5, atol=1e-13)
    # the four-point kernel gives a different (but also unit-sum) interpolation
    g4 = Grid(n, [v / n[0] for v in n])
    assert not np.allclose(ib.interp(g4, q, v), ib.interp(g, q, v))
    assert peskin.phi(np.array([0.0]))[0] != bkp6.phi(np.array([0.0]))[0]
