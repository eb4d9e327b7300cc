"""Pins for the free-kinematics oracle (bodies under given force/torque).

* Dense bordered LU of the enlarged system == DFT Schur route.
* Reciprocity: the velocities a free body takes under load F, imposed as
  prescribed velocities, give back exactly the load F = K^T Lambda; the
  resistance matrix K^T M^-1 K is symmetric positive definite.
* Zero load on a lone free body gives the zero solution.
"""
import numpy as np
import pytest

from oracle import fft_stokes
from oracle.free import FreeProblem, resistance, solve_free_fft
from oracle.system import drag
from synthetic import small_2d, small_3d

from ._util import oracle_problem


def _fp(wl, free):
    return FreeProblem(oracle_problem(wl), free)


CASES = [
    ("2d_two_free", lambda: small_2d(12, nbody=2, seed=3), [True, True]),
    ("2d_free_and_prescribed", lambda: small_2d(12, nbody=2, seed=4), [True, False]),
    ("3d_one_free", lambda: small_3d(8), [True]),
]


@pytest.mark.parametrize("name,mk,free", CASES)
def test_free_dense_equals_fft(name, mk, free):
    wl = mk()
    fp = _fp(wl, free)
    UO = wl.UO()
    b = fp.rhs(UO)
    x = fp.solve_dense(b)
    assert fp.residual(x, b) < 1e-10
    v, p, lam, U = solve_free_fft(fp, UO)
    xf = fp.join(v, p, lam, U)
    assert np.linalg.norm(x - xf) / np.linalg.norm(x) < 1e-10
    # force balance on every free body
    FT = drag(fp.p, lam)
    assert np.allclose(FT[fp.free], UO[fp.free], rtol=1e-10, atol=1e-12)


def test_reciprocity_and_resistance_spd():
    wl = small_2d(12, nbody=2, seed=3)
    fp = _fp(wl, [True, True])
    R = resistance(fp)
    assert np.allclose(R, R.T, rtol=1e-10, atol=1e-12 * np.abs(R).max())
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() > 0
    F = wl.UO()
    v, p, lam, U = solve_free_fft(fp, F)
    assert np.allclose(R @ U, F.ravel(), rtol=1e-9, atol=1e-12)
    # the free velocities imposed as prescribed ones reproduce the load
    vp, pp, lamp = fft_stokes.solve_coupled(fp.p, U.reshape(2, -1))
    assert np.allclose(drag(fp.p, lamp), F, rtol=1e-9, atol=1e-12)
    assert np.allclose(lamp, lam, rtol=1e-8, atol=1e-12)


def test_zero_load_zero_motion():
    wl = small_3d(8)
    fp = _fp(wl, [True])
    b = fp.rhs(np.zeros((1, 6)))
    assert not b.any()
    v, p, lam, U = solve_free_fft(fp, np.zeros((1, 6)))
    assert np.abs(U).max() == 0.0 and np.abs(lam).max() == 0.0
