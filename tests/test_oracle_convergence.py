"""First-order convergence of the oracle's constrained solve to an analytic
flow (CPU).

Sec. VII.C checks the method against concentric shells with an exact
solution and finds the velocity error falling about linearly with h (Table
v_errors).  The 2-D analogue used here: a rigid disk of radius R1 spinning
at omega inside a fixed rigid ring of radius R2, both represented only by
their boundary markers (spacing 2h) in a periodic box of steady Stokes flow.
The exact flow is rigid rotation inside the disk, circular Couette flow
v_theta = A r + B / r between the two (A = -omega R1^2 / (R2^2 - R1^2),
B = omega R1^2 R2^2 / (R2^2 - R1^2)), and rest outside the ring.  The
oracle's velocity (exact Schur solve by the DFT, Sec. III.C) is compared with
it on every face of the box; the relative L2 error must halve with h.

A sign slip in the rigid-body map, a dropped spreading term or a transposed
operand leaves an O(1) error that does not converge, and fails here.
"""
import numpy as np
import pytest

from oracle import fft_stokes
from oracle.mac import Grid
from oracle.system import Problem
from synthetic import disk_markers

R1, R2, OMEGA = 0.15, 0.35, 1.0


def couette_error(n):
    h = 1.0 / n
    inner, outer = disk_markers(R1, h), disk_markers(R2, h)
    c = np.array([0.5, 0.5])
    q = np.concatenate([c + inner, c + outer])
    rel = np.concatenate([inner, outer])
    body = np.array([0] * len(inner) + [1] * len(outer))
    g = Grid((n, n))
    pr = Problem(g, q, rel, body, 2)
    v, _, _ = fft_stokes.solve_coupled(pr, np.array([[0.0, 0.0, OMEGA], [0.0, 0.0, 0.0]]))
    A = -OMEGA * R1 ** 2 / (R2 ** 2 - R1 ** 2)
    B = OMEGA * R1 ** 2 * R2 ** 2 / (R2 ** 2 - R1 ** 2)
    err2 = ref2 = 0.0
    for a in range(2):
        X, Y = g.face_coords(a)
        dx, dy = X - 0.5, Y - 0.5
        r = np.maximum(np.hypot(dx, dy), 1e-300)
        vt = np.where(r < R1, OMEGA * r, np.where(r < R2, A * r + B / r, 0.0))
        exact = -vt * dy / r if a == 0 else vt * dx / r
        err2 += np.sum((v[a] - exact) ** 2)
        ref2 += np.sum(exact ** 2)
    return np.sqrt(err2 / ref2)


def test_rotating_disk_in_ring_converges_first_order():
    errs = [couette_error(n) for n in (32, 64, 128)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 0.06, errs
    for p in orders:
        assert 0.85 < p < 1.3, (errs, orders)


@pytest.mark.slow
def test_rotating_disk_in_ring_256():
    e128, e256 = couette_error(128), couette_error(256)
    assert 0.9 < np.log2(e128 / e256) < 1.2
