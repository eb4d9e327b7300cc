"""Fluid-marker coupling and rigid-body kinematics.

Interpolation and spreading (Sec. III.A):
  (J v)_i^alpha = sum_k v_k^alpha  prod_beta phi((q_i - r_k^alpha)_beta / h)
  (S L)_k^alpha = h^-d sum_i L_i^alpha prod_beta phi((q_i - r_k^alpha)_beta / h)
  J = S* = h^d S^T                          (Sec. III.A, adjointness)
Periodic steady Stokes spreads S~ = S - vol^-1 1^T (Sec. III.D,
Eq. constrained_periodic): the total marker force is removed as a uniform
force density.

Rigid-body map K (Sec. II; the body moves with linear velocity U and angular
velocity Omega about its reference point X):
  (K [U; Omega])_i = U + Omega x (q_i - X)     (2-D: Omega x r = omega (-r_y, r_x))
  K^T Lambda       = [sum_i Lambda_i ; sum_i (q_i - X) x Lambda_i]
and the constraint row of Eq. constrained_Stokes reads -J v = W with
W = -K U (the markers move rigidly, J v = K U).

Body orientation (Sec. II): a body's markers sit at q_i = X + Q(q) r_i with
r_i given in the body frame and Q(q) the rotation of the unit quaternion q
(``quat_rotate``).
"""
import numpy as np

from . import bkp6, peskin


def kernel_module(grid):
    """the 1-D kernel of the grid's regularised delta: the 4-point Peskin
    kernel, or the six-point kernel of Bao, Kaye and Peskin"""
    return bkp6 if getattr(grid, "kernel", "peskin4") == "bkp6" else peskin


def kernel_width(grid):
    return 6 if getattr(grid, "kernel", "peskin4") == "bkp6" else 4


def _stencil(grid, q, alpha):
    """Per-axis node windows and weights for component alpha.

    Returns a list over axes beta of (nodes[N,W] wrapped mod n_beta, w[N,W]),
    W = 4 or 6 the kernel's support.  Face i of component alpha sits at
    (i_beta + 1/2 - delta_{alpha beta}/2) h.
    """
    out = []
    kw = kernel_width(grid)
    for b in range(grid.d):
        off = 0.0 if b == alpha else 0.5
        s = q[:, b] / grid.h - off
        j0, w = kernel_module(grid).support_weights(s)
        nodes = (j0[:, None] + np.arange(kw)) % grid.n[b]
        out.append((nodes, w))
    return out


def _tensor_iter(grid, st):
    """Yield (flat_index[N], weight[N]) over the W^d tensor-product support."""
    d = grid.d
    import itertools

    for combo in itertools.product(range(kernel_width(grid)), repeat=d):
        flat = np.zeros(st[0][0].shape[0], dtype=np.int64)
        w = np.ones(st[0][0].shape[0])
        stride = 1
        for b in range(d):
            flat = flat + st[b][0][:, combo[b]] * stride
            w = w * st[b][1][:, combo[b]]
            stride *= grid.n[b]
        yield flat, w


def interp(grid, q, v):
    """J v: velocity field (list of d arrays) -> marker velocities [N, d]."""
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros((q.shape[0], grid.d))
    for a in range(grid.d):
        va = v[a].ravel()
        st = _stencil(grid, q, a)
        for flat, w in _tensor_iter(grid, st):
            out[:, a] += w * va[flat]
    return out


def spread(grid, q, lam):
    """S Lambda: marker forces [N, d] -> face force density (list of d arrays)."""
    q = np.asarray(q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    out = []
    for a in range(grid.d):
        f = np.zeros(grid.ncell)
        st = _stencil(grid, q, a)
        for flat, w in _tensor_iter(grid, st):
            np.add.at(f, flat, w * lam[:, a])
        out.append((f / grid.h ** grid.d).reshape(grid.shape))
    return out


def spread_tilde(grid, q, lam):
    """S~ Lambda = S Lambda - vol^-1 sum_i Lambda_i (periodic steady Stokes,
    Eq. constrained_periodic); plain S otherwise."""
    f = spread(grid, q, lam)
    if grid.steady:
        tot = np.asarray(lam).sum(axis=0)
        f = [f[a] - tot[a] / grid.vol for a in range(grid.d)]
    return f


def interp_bruteforce(grid, q, v):
    """J v written as the full sum over every face with minimum-image
    distances (no support window): O(N * cells), for tiny grids only."""
    q = np.asarray(q, dtype=np.float64)
    out = np.zeros((q.shape[0], grid.d))
    for a in range(grid.d):
        coords = grid.face_coords(a)
        for i in range(q.shape[0]):
            w = np.ones(grid.shape)
            for b in range(grid.d):
                dx = q[i, b] - coords[b]
                dx = dx - grid.L[b] * np.round(dx / grid.L[b])
                w = w * kernel_module(grid).phi(dx / grid.h)
            out[i, a] = np.sum(w * v[a])
    return out


def n_rot(d):
    return 1 if d == 2 else 3


def _hamilton(p, q):
    """Quaternion product p q of (w, x, y, z) quaternions (rows of [..., 4])."""
    pw, px, py, pz = p
    qw, qx, qy, qz = q
    return np.array([pw * qw - px * qx - py * qy - pz * qz,
                     pw * qx + px * qw + py * qz - pz * qy,
                     pw * qy - px * qz + py * qw + pz * qx,
                     pw * qz + px * qy - py * qx + pz * qw])


def quat_rotate(quat, r):
    """Lab-frame offsets Q(q) r_i of body-frame offsets r[N, 3] (Sec. II: the
    body's orientation; the marker positions are q_i = X + Q(q) r_i).

    Written from the definition of a rotation by a unit quaternion: the pure
    quaternion (0, r) is conjugated, q (0, r) q^*, one marker at a time; the
    quaternion is normalised first."""
    qq = np.asarray(quat, dtype=np.float64)
    qq = qq / np.sqrt(np.sum(qq * qq))
    conj = qq * np.array([1.0, -1.0, -1.0, -1.0])
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(r)
    for i in range(r.shape[0]):
        pure = np.array([0.0, r[i, 0], r[i, 1], r[i, 2]])
        out[i] = _hamilton(_hamilton(qq, pure), conj)[1:]
    return out


def apply_K(rel, body, UO, d):
    """K: per-body rigid velocities UO[B, d + rot] -> marker velocities [N, d].

    rel[N, d] = q_i - X_body(i) (unwrapped), body[N] = body index of marker i.
    """
    rel = np.asarray(rel, dtype=np.float64)
    UO = np.asarray(UO, dtype=np.float64).reshape(-1, d + n_rot(d))
    U = UO[body, :d]
    Om = UO[body, d:]
    if d == 2:
        w = Om[:, 0]
        return U + np.stack([-w * rel[:, 1], w * rel[:, 0]], axis=1)
    return U + np.cross(Om, rel)


def apply_KT(rel, body, lam, d, nbody):
    """K^T: marker forces [N, d] -> per-body [force; torque] [B, d + rot]."""
    rel = np.asarray(rel, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    out = np.zeros((nbody, d + n_rot(d)))
    for i in range(lam.shape[0]):
        b = body[i]
        out[b, :d] += lam[i]
        if d == 2:
            out[b, 2] += rel[i, 0] * lam[i, 1] - rel[i, 1] * lam[i, 0]
        else:
            out[b, 3:] += np.cross(rel[i], lam[i])
    return out


def J_matrix(grid, q):
    """J as a dense (N*d) x (d*ncell) matrix (marker-major rows i*d + alpha)."""
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[0]
    Jm = np.zeros((N * grid.d, grid.d * grid.ncell))
    for a in range(grid.d):
        st = _stencil(grid, q, a)
        for flat, w in _tensor_iter(grid, st):
            for i in range(N):
                Jm[i * grid.d + a, a * grid.ncell + flat[i]] += w[i]
    return Jm
