"""Approximate marker mobility M~ (Sec. IV, Eq. M_tilde_ij).

  M~_ij = f(r_ij) I + g(r_ij) r^_ij (x) r^_ij,   r_ij = q_i - q_j

built block-diagonally, one dense (d N_b) x (d N_b) block per body (Sec. VIII:
the mobility of several bodies is approximated body by body).

3-D steady Stokes: the RPY tensor (Eq. RPYTensor) with hydrodynamic radius a
(a = 1.25 h for the 4-point kernel, Sec. IV.A footnote), and the periodic
correction of App. A, f <- f - 2.84 / (6 pi eta l), applied to every entry of
f (the self term included, as for the periodic Stokes drag of a sphere).

2-D steady Stokes (App. B, Eqs. fg_tilde_Stokes_2d and fg_steady_2d):
  f(r) = f(0) - f~(r/h) / (4 pi eta),   g(r) = g~(r/h) / (4 pi eta),
  f(0) = ln(l / (3.708 a)) / (4 pi eta),  g(0) = 0,
  f~(x) = (a0 x^2 + a1 x^3 + a2 x^3 ln x) / (1 + a3 x + a4 x^2 + a2 x^3)
  g~(x) = (b0 x^2 + b1 x^3) / (1 + b2 x + b3 x^2 + b1 x^3)
with the coefficients passed in (the paper does not print them).
"""
import numpy as np


def rpy_fg(r, a, eta):
    """RPY f(r), g(r) (Eq. RPYTensor)."""
    r = np.asarray(r, dtype=np.float64)
    c = 1.0 / (6.0 * np.pi * eta * a)
    far = r > 2.0 * a
    rs = np.where(far, r, 1.0)
    f = np.where(far, c * (0.75 * a / rs + 0.5 * a ** 3 / rs ** 3), c * (1.0 - 9.0 * r / (32.0 * a)))
    g = np.where(far, c * (0.75 * a / rs - 1.5 * a ** 3 / rs ** 3), c * (3.0 * r / (32.0 * a)))
    return f, g


def fg_2d_steady(r, h, eta, l, a, coef):
    """App. B steady 2-D f(r), g(r); coef = (a0..a4, b0..b3)."""
    a0, a1, a2, a3, a4, b0, b1, b2, b3 = [float(c) for c in coef]
    r = np.asarray(r, dtype=np.float64)
    x = r / h
    xs = np.where(x > 0, x, 1.0)
    lnx = np.where(x > 0, np.log(xs), 0.0)
    ft = (a0 * x ** 2 + a1 * x ** 3 + a2 * x ** 3 * lnx) / (1.0 + a3 * x + a4 * x ** 2 + a2 * x ** 3)
    gt = (b0 * x ** 2 + b1 * x ** 3) / (1.0 + b2 * x + b3 * x ** 2 + b1 * x ** 3)
    f0 = np.log(l / (3.708 * a)) / (4.0 * np.pi * eta)
    return f0 - ft / (4.0 * np.pi * eta), gt / (4.0 * np.pi * eta)


def mtilde_block(rel, fg):
    """Dense d N x d N block from pair functions fg(r) -> (f, g)."""
    rel = np.asarray(rel, dtype=np.float64)
    N, d = rel.shape
    M = np.zeros((N * d, N * d))
    for i in range(N):
        for j in range(N):
            rv = rel[i] - rel[j]
            r = np.sqrt(np.dot(rv, rv))
            f, g = fg(np.array(r))
            f = float(f)
            g = float(g)
            blk = f * np.eye(d)
            if r > 0:
                e = rv / r
                blk = blk + g * np.outer(e, e)
            M[i * d:(i + 1) * d, j * d:(j + 1) * d] = blk
    return M


def mtilde_3d_rpy(rel, h, eta, l, a_over_h=1.25, periodic=True):
    a = a_over_h * h
    corr = 2.84 / (6.0 * np.pi * eta * l) if periodic else 0.0

    def fg(r):
        f, g = rpy_fg(r, a, eta)
        return f - corr, g

    return mtilde_block(rel, fg)


def mtilde_2d_steady(rel, h, eta, l, a_over_h, coef):
    a = a_over_h * h
    return mtilde_block(rel, lambda r: fg_2d_steady(r, h, eta, l, a, coef))
