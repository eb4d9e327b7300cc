"""Pins for the oracle's tabulated pair mobility M~ (periodic grids), the
approximate mobility of the library's IBR_MOB_PAIR model.

  - Markers on one lattice of the grid (every q_i = x0 + integer multiples of
    h) and a single source point at x0: the periodic grid is invariant under
    lattice shifts, so the table reproduces the true mobility M = J L^-1 S~
    exactly (any transposed index, staggering or sign error breaks this).
  - Off the lattice: M~ is symmetric (to rounding), and close to M (the kernel's
    translation invariance, Sec. IV): the spectrum of M~^-1 M stays near 1.
"""
import numpy as np
import pytest

from oracle import fft_stokes, mobility
from oracle.mac import Grid
from oracle.system import Problem
from synthetic import disk_markers, sphere_markers


def _problem(n, d, q):
    g = Grid((n,) * d, (1.0,) * d, 1.0)
    q = np.mod(q, 1.0)
    N = q.shape[0]
    return g, Problem(g, q, q - q.mean(0), np.zeros(N, dtype=np.int64), 1)


@pytest.mark.parametrize("d,n", [(2, 32), (3, 12)])
def test_lattice_markers_reproduce_true_mobility(d, n):
    rng = np.random.default_rng(3)
    h = 1.0 / n
    x0 = (np.floor(0.5 * n) + rng.uniform(0.1, 0.9, d)) * h
    k = rng.integers(-4, 5, size=(7 if d == 2 else 5, d))
    k = np.unique(k, axis=0)
    q = x0[None, :] + k * h
    g, pr = _problem(n, d, q)
    M = fft_stokes.mobility_true(pr)
    Mt = mobility.pair_table_mtilde(g, pr.q, [x0])
    assert np.abs(Mt - M).max() < 1e-12 * np.abs(M).max()


@pytest.mark.parametrize("d,n", [(2, 48), (3, 16)])
def test_off_lattice_symmetric_and_close_to_true(d, n):
    h = 1.0 / n
    c = np.full(d, 0.5) + 0.37 * h
    rel = disk_markers(0.15, h) if d == 2 else sphere_markers(3.0 * h, 24)
    g, pr = _problem(n, d, c + rel)
    M = fft_stokes.mobility_true(pr)
    Mt = mobility.pair_table_mtilde(g, pr.q, mobility.pair_sources(g.n, h, d))
    assert np.abs(Mt - Mt.T).max() <= 1e-14 * np.abs(Mt).max()
    lam = np.linalg.eigvals(np.linalg.solve(Mt, M)).real
    assert lam.min() > 0.5 and lam.max() < 2.0, (lam.min(), lam.max())
    assert np.linalg.norm(Mt - M) < 0.1 * np.linalg.norm(M)


def test_pair_sources_are_off_the_nodes():
    for x0 in mobility.pair_sources((32, 32), 1.0 / 32, 2):
        fr = x0 * 32 - np.floor(x0 * 32)
        assert np.all(fr > 0.2) and np.all(fr < 0.8)
