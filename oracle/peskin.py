"""The 4-point Peskin kernel (Sec. III.A; the kernel of the paper's ref.
IBM_PeskinReview, Peskin 2002, Eq. 6.27 there).

phi is a function of a distance measured in grid units r/h.  It is the unique
continuous function with support [-2, 2] that satisfies, for every real shift s,

  sum_j phi(s - j)             = 1        (partition of unity)
  sum_j (s - j) phi(s - j)     = 0        (first moment)
  sum_{j even} phi(s - j)      = 1/2      (even-odd condition)
  sum_j phi(s - j)^2           = 3/8      (sum of squares)

``phi`` evaluates Peskin's published closed form of that function (the
roots of the quadratic the conditions give on each unit interval); the tests
check the four conditions themselves by brute force over many shifts.
"""
import numpy as np


def phi(r):
    """4-point Peskin kernel evaluated at r (grid units), float64, vectorised."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    inner = r < 1.0
    outer = (r >= 1.0) & (r < 2.0)
    ri = r[inner]
    out[inner] = (3.0 - 2.0 * ri + np.sqrt(1.0 + 4.0 * ri - 4.0 * ri * ri)) / 8.0
    ro = r[outer]
    out[outer] = (5.0 - 2.0 * ro - np.sqrt(-7.0 + 12.0 * ro - 4.0 * ro * ro)) / 8.0
    return out


def support_weights(s):
    """The 4 nodes j = floor(s)-1 .. floor(s)+2 and weights phi(s - j).

    ``s`` is a position in grid units measured from node 0.  Nodes outside
    this window have |s - j| >= 2 and weight zero.  Returns (j0, w[...,4]).
    """
    s = np.asarray(s, dtype=np.float64)
    j0 = np.floor(s).astype(np.int64) - 1
    offs = np.arange(4)
    w = phi(s[..., None] - (j0[..., None] + offs))
    return j0, w
