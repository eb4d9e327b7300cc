"""Seeded marker geometries and problem descriptions.

Shapes follow the paper's workloads: surface ("shell") markers at a spacing
of about 2h (Sec. VI, s/h ~ 2), disks in 2-D (Sec. VII.E) and spheres in 3-D
(Sec. VII.A, VII.G).  Seeds default to 1505 + the workload number.
"""
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "disk_markers",
    "sphere_markers",
    "Body",
    "Workload",
    "disk_64",
    "sphere_128",
    "small_2d",
    "small_3d",
    "random_velocities",
]


def disk_markers(radius, h, spacing=2.0):
    """N = round(2 pi r / (spacing h)) points equally spaced on a circle,
    the first at angle 0; body-frame offsets [N, 2]."""
    N = max(3, int(round(2.0 * np.pi * radius / (spacing * h))))
    th = 2.0 * np.pi * np.arange(N) / N
    return np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)


def sphere_markers(radius, N):
    """N golden-spiral (Fibonacci) points on a sphere; body-frame offsets [N, 3]."""
    i = np.arange(N, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / N
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = np.pi * (3.0 - np.sqrt(5.0))
    ph = ga * i
    return radius * np.stack([rho * np.cos(ph), rho * np.sin(ph), z], axis=1)


@dataclass
class Body:
    center: np.ndarray          # [d]
    rel: np.ndarray             # [N_b, d] body-frame marker offsets (identity rotation)
    UO: np.ndarray              # [d + rot] prescribed linear + angular velocity


@dataclass
class Workload:
    name: str
    n: tuple                    # cells per axis, x first
    L: tuple
    eta: float = 1.0
    rho: float = 0.0
    dt: float = 0.0
    bodies: list = field(default_factory=list)
    tol: float = 1e-8

    @property
    def d(self):
        return len(self.n)

    def markers(self):
        """(q[N,d] lab positions, rel[N,d], body[N]) concatenated over bodies."""
        qs, rels, ids = [], [], []
        for b, body in enumerate(self.bodies):
            qs.append(body.center[None, :] + body.rel)
            rels.append(body.rel)
            ids.append(np.full(body.rel.shape[0], b, dtype=np.int64))
        return np.concatenate(qs), np.concatenate(rels), np.concatenate(ids)

    def UO(self):
        return np.stack([b.UO for b in self.bodies])


def random_velocities(rng, d, nbody):
    rot = 1 if d == 2 else 3
    return rng.standard_normal((nbody, d + rot))


def disk_64():
    """Periodic unit square, 64^2 MAC grid, eta = 1, steady Stokes; one disk of
    radius 0.1 at (0.5, 0.5) with 20 markers at ~2h; U = (1, 0), omega = 0."""
    h = 1.0 / 64
    rel = disk_markers(0.1, h)
    body = Body(np.array([0.5, 0.5]), rel, np.array([1.0, 0.0, 0.0]))
    return Workload("disk_64x64_periodic_stokes", (64, 64), (1.0, 1.0), bodies=[body], tol=1e-10)


def sphere_128(seed=1505 + 3, N=500):
    """Periodic unit cube, 128^3 MAC grid, eta = 1, steady Stokes; one sphere of
    radius 0.1 at the centre with 500 golden-spiral markers; U, Omega ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    rel = sphere_markers(0.1, N)
    UO = random_velocities(rng, 3, 1)[0]
    body = Body(np.array([0.5, 0.5, 0.5]), rel, UO)
    return Workload("sphere_128^3_periodic_stokes", (128, 128, 128), (1.0, 1.0, 1.0), bodies=[body], tol=1e-8)


def small_2d(n=16, nbody=1, seed=7, rho=0.0, dt=0.0, radius_h=2.5, shift=(0.0, 0.0)):
    """Tiny periodic 2-D problem for dense checks: disks of radius radius_h*h,
    markers at ~2h, centres at seeded off-grid positions."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    bodies = []
    for b in range(nbody):
        c = np.array([(b + 0.5) / nbody, 0.5]) + np.array(shift) + rng.uniform(-0.5, 0.5, 2) * h
        rel = disk_markers(radius_h * h, h)
        bodies.append(Body(c, rel, random_velocities(rng, 2, 1)[0]))
    return Workload(f"small2d_{n}", (n, n), (1.0, 1.0), rho=rho, dt=dt, bodies=bodies, tol=1e-10)


def small_3d(n=8, N=12, seed=11, rho=0.0, dt=0.0, radius_h=1.6):
    """Tiny periodic 3-D problem for dense checks."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    c = np.array([0.5, 0.5, 0.5]) + rng.uniform(-0.5, 0.5, 3) * h
    rel = sphere_markers(radius_h * h, N)
    body = Body(c, rel, random_velocities(rng, 3, 1)[0])
    return Workload(f"small3d_{n}", (n, n, n), (1.0, 1.0, 1.0), rho=rho, dt=dt, bodies=[body], tol=1e-10)
