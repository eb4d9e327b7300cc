"""The six-point kernel of Bao, Kaye and Peskin (the paper's ref.
New6ptKernel; Sec. III.A uses it: support of 6 grid points per direction,
three continuous derivatives, much better translational invariance than the
four-point kernel).

The paper does not print the kernel.  It is the function phi with support
[-3, 3] fixed by these conditions, for every shift r (grid units), with the
sums over all integers j:

  sum_j phi(r - j)               = 1        (zeroth moment)
  sum_j (-1)^j phi(r - j)        = 0        (even-odd: the even and the odd
                                             nodes each carry half)
  sum_j (r - j) phi(r - j)       = 0        (first moment)
  sum_j (r - j)^2 phi(r - j)     = K        (second moment: a constant)
  sum_j (r - j)^3 phi(r - j)     = 0        (third moment)
  sum_j phi(r - j)^2             = C        (sum of squares: a constant)

with K = 59/60 - sqrt(29)/20, the value for which phi has three continuous
derivatives, and C fixed by continuity at the integers: at r = 0 the nodes
+-3 lie on the edge of the support, so the five linear conditions determine
phi(0), phi(+-1), phi(+-2) and C is their sum of squares.

For a shift r in [0, 1) the six weights phi(r - j), j = -2 .. 3, are the
unknowns: the five linear conditions leave a one-parameter family
p(t) = p0 + t z (z spanning the null space), and the sum of squares picks t
from a quadratic; of its two roots the one that joins continuously with the
values at r = 0 is taken.  Everything here is computed from these
conditions by plain linear algebra in float64 (no closed form, no table).
"""
import numpy as np

K = 59.0 / 60.0 - np.sqrt(29.0) / 20.0
_JS = np.arange(-2, 4)  # node offsets j of the six weights phi(r - j)


def _at_zero():
    """phi(0), phi(1) = phi(-1), phi(2) = phi(-2) from the linear conditions
    at r = 0 (phi(+-3) = 0 there), and C = their sum of squares."""
    js = np.arange(-2, 3)
    A = np.stack([np.ones(5), (-1.0) ** js, -js, js ** 2.0, -(js ** 3.0)])
    b = np.array([1.0, 0.0, 0.0, K, 0.0])
    p = np.linalg.solve(A, b)
    return p, float(np.sum(p * p))


P0, C = _at_zero()


def weights(r):
    """The six weights phi(r - j), j = -2..3, for shifts r in [0, 1); r may
    be an array (result [..., 6])."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.zeros(r.shape + (6,))
    for idx in np.ndindex(r.shape):
        x = r[idx] - _JS  # the arguments r - j
        A = np.stack([np.ones(6), (-1.0) ** _JS, x, x ** 2, x ** 3])
        b = np.array([1.0, 0.0, 0.0, K, 0.0])
        p0 = np.linalg.lstsq(A, b, rcond=None)[0]
        z = np.linalg.svd(A)[2][-1]
        # |p0 + t z|^2 = C  ->  (z.z) t^2 + 2 (p0.z) t + (p0.p0 - C) = 0
        qa, qb, qc = z @ z, 2.0 * (p0 @ z), p0 @ p0 - C
        disc = max(qb * qb - 4.0 * qa * qc, 0.0)
        roots = [(-qb + sgn * np.sqrt(disc)) / (2.0 * qa) for sgn in (1.0, -1.0)]
        cands = [p0 + t * z for t in roots]
        out[idx] = min(cands, key=lambda p: _branch_distance(r[idx], p))
    return out


def _branch_distance(r, p):
    """distance from the r = 0 values, continued along r: the branch whose
    weights at r -> 0 approach (0, phi(2), phi(1), phi(0), phi(1), phi(2))
    in the order j = -2..3 is phi's (the sum of squares is the same on both;
    the other root is the mirror image through the midpoint)"""
    ref = np.array([P0[0], P0[1], P0[2], P0[3], P0[4], 0.0])  # j = -2..3 at r = 0
    mirrored = np.array([0.0, P0[0], P0[1], P0[2], P0[3], P0[4]])  # the r -> 1 limit
    w = 1.0 - r
    return np.sum((p - (w * ref + (1.0 - w) * mirrored)) ** 2)


def phi(x):
    """phi(x), x in grid units (vectorised)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    inside = np.abs(x) < 3.0
    xi = x[inside]
    fl = np.floor(xi)
    r = xi - fl
    j = (-fl).astype(np.int64)  # x = r - j
    w = weights(r)
    out[inside] = w[np.arange(xi.size), j + 2]
    return out


def support_weights(s):
    """The 6 nodes j = floor(s)-2 .. floor(s)+3 and weights phi(s - j) for
    positions s in grid units measured from node 0: (j0, w[..., 6])."""
    s = np.asarray(s, dtype=np.float64)
    j0 = np.floor(s).astype(np.int64) - 2
    r = s - np.floor(s)
    w = weights(r)  # node j0 + m carries phi(s - j0 - m) = phi(r - (m - 2)), the weight of j = m - 2
    return j0, w.reshape(s.shape + (6,))
