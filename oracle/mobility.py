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

Periodic grids, tabulated pair mobility (Sec. IV: the mobility of two markers
is, up to a small dependence on their position relative to the grid, a
function of their displacement; here that function is taken from the grid
itself instead of a fitted form): with T_s(r)^{ab} = (J(x0_s + r) L^-1 S~
e_b delta_{x0_s})_a the velocity at x0_s + r due to a unit force e_b at the
source point x0_s,
  M~_ij^{ab} = (1/2S) sum_s [ T_s(q_i - q_j)^{ab} + T_s(q_j - q_i)^{ba} ].
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


def mtilde_block(rel, fg, box=None):
    """Dense d N x d N block from pair functions fg(r) -> (f, g) (Eq.
    M_tilde_ij: every marker pair).  box: periodic lengths per axis (0 for a
    wall axis); displacements are then the minimum images."""
    rel = np.asarray(rel, dtype=np.float64)
    N, d = rel.shape
    M = np.zeros((N * d, N * d))
    for i in range(N):
        for j in range(N):
            rv = rel[i] - rel[j]
            if box is not None:
                for a in range(d):
                    if box[a] > 0:
                        rv[a] -= box[a] * np.round(rv[a] / box[a])
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


def mtilde_3d_rpy(rel, h, eta, l, a_over_h=1.25, periodic=True, box=None):
    a = a_over_h * h
    corr = 2.84 / (6.0 * np.pi * eta * l) if periodic else 0.0

    def fg(r):
        f, g = rpy_fg(r, a, eta)
        return f - corr, g

    return mtilde_block(rel, fg, box)


def mtilde_2d_steady(rel, h, eta, l, a_over_h, coef, box=None):
    a = a_over_h * h
    return mtilde_block(rel, lambda r: fg_2d_steady(r, h, eta, l, a, coef), box)


def pair_table_mtilde(grid, q, x0s):
    """Dense (d N)^2 M~ from the tabulated periodic pair mobility of the grid
    (exact DFT Stokes solves, one per source point and force direction)."""
    from . import fft_stokes, ib

    q = np.asarray(q, dtype=np.float64)
    N, d = q.shape
    L = np.array(grid.L, dtype=np.float64)
    M = np.zeros((N * d, N * d))
    for x0 in x0s:
        x0 = np.asarray(x0, dtype=np.float64)
        fields = []
        for b in range(d):
            lam = np.zeros((1, d))
            lam[0, b] = 1.0
            v, _ = fft_stokes.stokes_solve(grid, ib.spread_tilde(grid, x0[None, :], lam))
            fields.append(v)
        for i in range(N):
            for j in range(N):
                for r, tr in ((q[i] - q[j], False), (q[j] - q[i], True)):
                    p = np.mod(x0 + r, L)[None, :]
                    for b in range(d):
                        u = ib.interp(grid, p, fields[b])[0]  # T(r)[:, b]
                        for a in range(d):
                            if tr:
                                M[i * d + b, j * d + a] += u[a]
                            else:
                                M[i * d + a, j * d + b] += u[a]
    return M / (2.0 * len(x0s))


def pair_sources(n, h, d):
    """The two source points of the library's pair table: cell floor(n/2)
    along each axis, sub-cell offsets (0.3, 0.7, 0.45) h and (0.7, 0.3, 0.55) h."""
    fr = ((0.3, 0.7, 0.45), (0.7, 0.3, 0.55))
    return [np.array([(np.floor(0.5 * n[a]) + fr[k][a]) * h for a in range(d)]) for k in range(2)]
