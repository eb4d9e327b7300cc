"""Shared test helpers: build the same seeded problem for the GPU library
(through the C ABI) and for the oracle.  Both sides take their geometry from
``synthetic``; no numerical routine is shared."""
import numpy as np

from oracle import walls as W
from oracle.mac import Grid
from oracle.system import Problem


def oracle_problem(wl):
    q, rel, body = wl.markers()
    g = Grid(wl.n, wl.L, wl.eta, wl.rho, wl.dt, kernel=wl.kernel)
    q = np.mod(q, np.array(wl.L))
    return Problem(g, q, rel, body, len(wl.bodies))


def gpu_grid(abi, wl, precision, free=None, data=None):
    """free: optional list of flags, True for a body under given force/torque.
    data: optional {(axis, side): values [d, face points...]} wall velocities
    (those sides become IBR_VELOCITY walls; the other wall sides no-slip)."""
    bc = []
    for a, w in enumerate(wl.wall_flags()):
        for s in (0, 1):
            if not w:
                bc.append(abi.PERIODIC)
            else:
                bc.append(abi.VELOCITY if data is not None and (a, s) in data else abi.NOSLIP)
    kernel = abi.KERNEL_BKP6 if wl.kernel == "bkp6" else abi.KERNEL_PESKIN4
    g = abi.create_grid(wl.d, wl.n, wl.L, bc=bc, eta=wl.eta, rho=wl.rho, dt=wl.dt, kernel=kernel,
                        precision=precision)
    if data is not None:
        for (a, s), val in data.items():
            abi.set_boundary_velocity(g, 2 * a + s, np.ascontiguousarray(val, dtype=np.float64).ravel())
    for i, b in enumerate(wl.bodies):
        kin = abi.FREE if (free is not None and free[i]) else abi.PRESCRIBED
        bid = abi.add_body(g, b.center, kinematics=kin)
        abi.set_markers(g, bid, b.rel)
    return g


def oracle_wall_problem(wl):
    """the wall-bounded oracle problem with the markers of wl (no wrapping)"""
    q, rel, body = wl.markers()
    wg = W.WallGrid(wl.n, wl.L, wl.wall_flags(), wl.eta, wl.rho, wl.dt)
    return W.WallProblem(wg, q), rel, body


def rel_err(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def flat_fields(v):
    return np.concatenate([np.asarray(x).ravel() for x in v])
