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
    "wall_2d",
    "wall_3d",
    "nozzle",
    "nozzle_walls",
    "parabolic_inflow",
    "ellipsoid_markers",
    "random_quaternion",
    "batch_2d",
    "serve_3d",
    "Request",
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
    walls: tuple = ()           # per axis: True for walls at both ends (empty: all periodic)
    kernel: str = "peskin4"     # regularised delta of J and S: "peskin4" or "bkp6" (six-point)

    @property
    def d(self):
        return len(self.n)

    def wall_flags(self):
        return tuple(bool(w) for w in self.walls) if self.walls else (False,) * self.d

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


def wall_2d(n=(24, 16), walls=(True, True), nbody=2, seed=31, rho=0.0, dt=0.0, radius_h=2.5):
    """Small 2-D box of height 1 (cells h = 1/n[1]) with walls on the flagged
    axes; disks of radius radius_h*h, markers at ~2h, one of them pushed
    into the kernel support of the low y-wall (and of the low x-wall when
    walls[0])."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n[1]
    L = (n[0] * h, 1.0)
    r = radius_h * h
    bodies = []
    for b in range(nbody):
        c = np.array([(b + 0.5) / nbody * L[0], 0.55]) + rng.uniform(-0.5, 0.5, 2) * h
        if b == 0:
            c[1] = r + rng.uniform(0.6, 1.4) * h
            if walls[0]:
                c[0] = r + rng.uniform(0.6, 1.4) * h
        bodies.append(Body(c, disk_markers(r, h), random_velocities(rng, 2, 1)[0]))
    return Workload(f"wall2d_{n[0]}x{n[1]}", tuple(n), L, rho=rho, dt=dt, bodies=bodies, tol=1e-10,
                    walls=tuple(walls))


def wall_3d(n=(8, 12, 8), walls=(False, True, True), seed=37, rho=0.0, dt=0.0, radius_h=1.6, N=12):
    """Small 3-D duct (height 1 along y) with walls on the flagged axes; one
    sphere of markers within the kernel support of the low y-wall."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n[1]
    L = tuple(m * h for m in n)
    r = radius_h * h
    c = np.array([0.5 * L[0], r + rng.uniform(0.6, 1.2) * h, 0.5 * L[2]]) + np.array([1, 0, 1]) * rng.uniform(-0.5, 0.5, 3) * h
    body = Body(c, sphere_markers(r, N), random_velocities(rng, 3, 1)[0])
    return Workload(f"wall3d_{n[0]}x{n[1]}x{n[2]}", tuple(n), L, rho=rho, dt=dt, bodies=[body], tol=1e-10,
                    walls=tuple(walls))


def nozzle_walls(h, depth=0.3, half_len=0.9, spacing=2.0, min_gap=1.0):
    """Marker rows of the two nozzle walls in the channel [0,2] x [0,1]: the
    upper wall y = 1 - depth (1 + cos(pi (x - 1) / half_len)) / 2 for
    |x - 1| <= half_len, the lower one its mirror image y -> 1 - y (throat
    [0.3, 0.7] for depth 0.3).  Markers at arc-length spacing `spacing` h,
    symmetric about x = 1; markers closer than min_gap h to the channel wall
    (where the nozzle wall merges with it) are left out: that wall already
    holds the fluid there, and a marker on it would give a zero constraint
    row.  Returns [(centre, rel)] for the upper and lower walls."""
    x = np.linspace(1.0 - half_len, 1.0 + half_len, 200001)
    y = 1.0 - depth * 0.5 * (1.0 + np.cos(np.pi * (x - 1.0) / half_len))
    seg = np.hypot(np.diff(x), np.diff(y))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    smid = s[-1] / 2.0
    k = np.arange(-int(smid / (spacing * h)), int(smid / (spacing * h)) + 1)
    sk = smid + k * spacing * h
    xs = np.interp(sk, s, x)
    ys = np.interp(sk, s, y)
    keep = (1.0 - ys) >= min_gap * h
    up = np.stack([xs[keep], ys[keep]], axis=1)
    lo = np.stack([xs[keep], 1.0 - ys[keep]], axis=1)
    out = []
    for q in (up, lo):
        c = q.mean(axis=0)
        out.append((c, q - c))
    return out


def parabolic_inflow(n1, U=1.0):
    """Normal velocity 4 U y (1 - y) at the cell-centred heights of a wall
    face column of a channel of height 1 with n1 cells."""
    y = (np.arange(n1) + 0.5) / n1
    return 4.0 * U * y * (1.0 - y)


def nozzle(n=(256, 128), Re=0.0, U=1.0, u_max=None):
    """2-D nozzle flow: channel [0,2] x [0,1], no-slip at y = 0, 1, parabolic
    inflow/outflow 4 U y (1 - y) at x = 0 and x = 2, two fixed rigid nozzle
    walls (nozzle_walls) forming a throat of width 0.4.  Re = rho U 0.4 / eta
    with rho = 1 (Re = 0: steady Stokes, eta = 1); the time step is
    0.5 h / u_max (u_max: the largest speed of the flow, e.g. of the steady
    Stokes solution; default U, the inflow peak)."""
    h = 1.0 / n[1]
    bodies = [Body(c, rel, np.zeros(3)) for c, rel in nozzle_walls(h)]
    if Re == 0:
        eta, rho, dt = 1.0, 0.0, 0.0
    else:
        eta, rho, dt = U * 0.4 / Re, 1.0, 0.5 * h / (U if u_max is None else u_max)
    return Workload(f"nozzle_{n[0]}x{n[1]}_Re{Re:g}", tuple(n), (2.0, 1.0), eta=eta, rho=rho, dt=dt, bodies=bodies,
                    tol=1e-8, walls=(True, True))


# ---------------------------------------------------------------------------
# batched and served problem mixes (independent periodic problems)

def ellipsoid_markers(b, aspect, h, spacing=2.2):
    """Golden-spiral points on a prolate ellipsoid with semi-axes
    (aspect b, b, b) along the body-frame x, y, z: a sphere's points scaled
    per axis, their number raised (from the sphere rule N = area / ((sqrt 3 / 2)
    (2h)^2)) until the largest nearest-neighbour distance is <= spacing h."""
    from scipy.spatial import cKDTree

    a = aspect * b
    if aspect > 1.0:
        e = np.sqrt(1.0 - (b / a) ** 2)
        area = 2.0 * np.pi * b * b * (1.0 + a / (b * e) * np.arcsin(e))
    else:
        area = 4.0 * np.pi * b * b
    N = max(12, int(round(area / (np.sqrt(3.0) / 2.0 * (2.0 * h) ** 2))))
    scale = np.array([a, b, b])
    while True:
        pts = sphere_markers(1.0, N) * scale
        dist, _ = cKDTree(pts).query(pts, k=2)
        if dist[:, 1].max() <= spacing * h or N > 200000:
            return pts
        N = int(N * 1.1) + 1


def random_quaternion(rng):
    """Uniformly distributed unit quaternion (w, x, y, z) (Shoemake's method)."""
    u1, u2, u3 = rng.uniform(size=3)
    q = np.array([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)])
    return np.array([q[3], q[0], q[1], q[2]])


@dataclass
class Request:
    """One independent periodic problem of a batch or a served stream: the
    unit box with n cells per axis, bodies given by centre, orientation and
    body-frame marker offsets, rigid velocities [B, d + rot]; t_arrival in s."""
    n: tuple
    centers: list
    quats: list
    rels: list
    UO: np.ndarray
    t_arrival: float = 0.0
    shapes: list = field(default_factory=list)

    @property
    def d(self):
        return len(self.n)

    @property
    def L(self):
        return (1.0,) * self.d

    @property
    def N(self):
        return int(sum(r.shape[0] for r in self.rels))

    def workload(self, rotate=None):
        """The same problem as a Workload, the body-frame offsets turned into
        lab-frame ones by rotate(quat, rel) (3-D; the caller supplies the
        rotation, this module holds geometry only)."""
        bodies = []
        for c, q, r, uo in zip(self.centers, self.quats, self.rels, self.UO):
            if self.d == 3 and rotate is None:
                raise ValueError("a 3-D request needs the rotation of its quaternions")
            rel = r if self.d == 2 else rotate(q, r)
            bodies.append(Body(np.asarray(c, dtype=np.float64), rel, np.asarray(uo)))
        return Workload(f"req_{'x'.join(map(str, self.n))}_{len(bodies)}b", tuple(self.n), self.L, bodies=bodies,
                        tol=1e-8)


def _periodic_gap(c1, c2):
    d = np.abs(np.asarray(c1) - np.asarray(c2))
    d = np.minimum(d, 1.0 - d)
    return float(np.sqrt((d * d).sum()))


def _place(rng, radii, d, gap, tries=2000):
    """Rejection-sampled centres in the periodic unit box with bounding
    circles/spheres at least `gap` apart; bodies that find no place in
    `tries` draws are dropped.  Returns the kept indices and centres."""
    keep, cs = [], []
    for i, r in enumerate(radii):
        for _ in range(tries):
            c = rng.uniform(0.0, 1.0, d)
            if all(_periodic_gap(c, c2) >= r + radii[j] + gap for j, c2 in zip(keep, cs)):
                keep.append(i)
                cs.append(c)
                break
    return keep, cs


def batch_2d(count=64, seed=1505 + 4, sizes=(64, 128, 256, 512)):
    """Independent 2-D periodic Stokes problems: n uniform over `sizes`
    (square unit box), 1 to 8 disks of radius U[0.05, 0.15] with markers at
    2h, non-overlapping with a gap >= 4h (the kernel support), rigid
    velocities N(0, 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        h = 1.0 / n
        nb = int(rng.integers(1, 9))
        radii = rng.uniform(0.05, 0.15, nb)
        keep, cs = _place(rng, radii, 2, 4.0 * h)
        rels = [disk_markers(radii[i], h) for i in keep]
        UO = random_velocities(rng, 2, len(keep))
        out.append(Request((n, n), cs, [np.array([1.0, 0, 0, 0])] * len(keep), rels, UO,
                           shapes=[("disk", radii[i]) for i in keep]))
    return out


def serve_3d(count=60, rate=50.0, seed=1505 + 5, sizes=(64, 96, 128, 192), max_bodies=16):
    """A stream of 3-D periodic Stokes requests with Poisson arrivals at
    `rate` per second: n uniform over `sizes`; 1 to max_bodies rigid bodies,
    each a sphere or a prolate ellipsoid (aspect U[1, 3], semi-minor axis
    U[0.05, 0.12], uniformly random orientation) carrying surface markers at
    <= 2.2h (ellipsoid_markers), non-overlapping with a gap >= 4h between
    bounding spheres; rigid velocities N(0, 1)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice(sizes))
        h = 1.0 / n
        nb = int(rng.integers(1, max_bodies + 1))
        aspect = np.where(rng.uniform(size=nb) < 0.5, 1.0, rng.uniform(1.0, 3.0, nb))
        b = rng.uniform(0.05, 0.12, nb)
        keep, cs = _place(rng, aspect * b, 3, 4.0 * h)
        quats = [random_quaternion(rng) for _ in keep]
        rels = [ellipsoid_markers(b[i], aspect[i], h) for i in keep]
        UO = random_velocities(rng, 3, len(keep))
        out.append(Request((n, n, n), cs, quats, rels, UO, t_arrival=t,
                           shapes=[("ellipsoid" if aspect[i] > 1 else "sphere", b[i], aspect[i]) for i in keep]))
    return out
