"""Exact periodic Stokes solves by the discrete Fourier transform.

On a periodic MAC grid every operator of ``mac`` is diagonal in the DFT basis
(Sec. III.C: "for a periodic system, the discrete operators commute",
Eq. L_inv_periodic).  With theta_alpha = 2 pi k_alpha / n_alpha and numpy's
forward transform (a shift i -> i-1 multiplies mode k by exp(-i theta)):

  G^alpha  ->  (1 - e^{-i theta_alpha}) / h
  D^alpha  ->  (e^{i theta_alpha} - 1) / h
  Lap      ->  -sum_beta 4 sin^2(theta_beta / 2)
  A        ->  a(k) = rho/dt + eta h^-2 sum_beta 4 sin^2(theta_beta/2)

so the unconstrained Stokes system (Eq. Stokes_saddle)
  A v + G pi = f,  -D v = hd
is solved mode by mode:  pi^ = (D^ f^ + a hd^) / (D^ G^),  v^ = (f^ - G^ pi^) / a.
At k = 0 the pressure is set to zero (<pi> = 0); for steady Stokes (a(0) = 0)
the mean velocity is zero (the restricted inverse of Sec. V.A, alpha = 1).

The exact coupled solution follows the Schur-complement route of Sec. III.C:
  v~ = L^-1 g (+ L_p^-1 h),   M = J L^-1 S~   (Eq. mob_def),
  M Lambda = -(W + J v~)      (Eq. lambda_sol),  v = v~ + L^-1 S~ Lambda.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import ib


def _symbols(grid):
    d = grid.d
    thetas = []
    for a in range(d):
        k = np.arange(grid.n[a])
        th = 2.0 * np.pi * k / grid.n[a]
        shape = [1] * d
        shape[grid.ax(a)] = grid.n[a]
        thetas.append(th.reshape(shape))
    Ghat = [(1.0 - np.exp(-1j * thetas[a])) / grid.h for a in range(d)]
    Dhat = [(np.exp(1j * thetas[a]) - 1.0) / grid.h for a in range(d)]
    s2 = sum(4.0 * np.sin(thetas[a] / 2.0) ** 2 for a in range(d))
    s2 = np.broadcast_to(s2, grid.shape)
    ahat = grid.sigma + grid.eta / grid.h ** 2 * s2
    DG = -s2 / grid.h ** 2
    return Ghat, Dhat, ahat, DG


def stokes_solve(grid, f, hd=None):
    """Exact solution (v, pi) of A v + G pi = f, -D v = hd on the periodic
    grid; for steady Stokes <f> must vanish and <v> = 0 is returned."""
    d = grid.d
    Ghat, Dhat, ahat, DG = _symbols(grid)
    fh = [np.fft.fftn(f[a]) for a in range(d)]
    hh = np.fft.fftn(hd) if hd is not None else np.zeros(grid.shape, dtype=complex)
    zero = tuple([0] * d)
    num = sum(Dhat[a] * fh[a] for a in range(d)) + ahat * hh
    DGs = DG.copy()
    DGs[zero] = 1.0
    ph = num / DGs
    ph[zero] = 0.0
    a_safe = ahat.copy()
    if grid.steady:
        a_safe[zero] = 1.0
    vh = [(fh[a] - Ghat[a] * ph) / a_safe for a in range(d)]
    if grid.steady:
        for a in range(d):
            vh[a][zero] = 0.0
    v = [np.real(np.fft.ifftn(vh[a])) for a in range(d)]
    p = np.real(np.fft.ifftn(ph))
    return v, p


def helmholtz_solve(grid, sigma, kappa, f):
    """Exact (sigma I - kappa h^-2 Lap) u = f on the periodic cell grid; for
    sigma == 0 the mean of f is ignored and <u> = 0 (the scalar operators of
    the V-cycles in P_S, Sec. V.B)."""
    _, _, _, DG = _symbols(grid)
    sym = sigma - kappa * DG  # DG = -h^-2 sum 4 sin^2
    zero = tuple([0] * grid.d)
    fh = np.fft.fftn(f)
    if sigma == 0.0:
        sym = sym.copy()
        sym[zero] = 1.0
        fh[zero] = 0.0
    return np.real(np.fft.ifftn(fh / sym))


def mobility_true(prob):
    """The true marker mobility M = J L^-1 S~ (Eq. mob_def), dense, formed
    column by column with exact DFT Stokes solves."""
    g = prob.grid
    dN = prob.N * g.d
    M = np.zeros((dN, dN))
    for j in range(dN):
        lam = np.zeros((prob.N, g.d))
        lam[j // g.d, j % g.d] = 1.0
        f = ib.spread_tilde(g, prob.q, lam)
        v, _ = stokes_solve(g, f)
        M[:, j] = ib.interp(g, prob.q, v).ravel()
    return M


def solve_coupled(prob, UO, g_force=None, h_div=None, dense_limit=3000, cg_tol=1e-13,
                  cg_maxiter=5000, return_info=False):
    """Exact (v, pi, Lambda) of the constrained system by the Schur route.

    M is formed densely when d*N <= dense_limit and solved by a symmetric
    solve; otherwise M Lambda = rhs is solved by conjugate gradients with one
    exact Stokes solve per product (M is SPD, Sec. III.C).
    """
    g = prob.grid
    d = g.d
    if g_force is None:
        g_force = [np.zeros(g.shape) for _ in range(d)]
    W = -ib.apply_K(prob.rel, prob.body, UO, d)
    vt, pt = stokes_solve(g, g_force, h_div)
    rhs = -(W + ib.interp(g, prob.q, vt)).ravel()
    info = {}
    if prob.N * d <= dense_limit:
        M = mobility_true(prob)
        lam = np.linalg.solve(M, rhs)
        info["method"] = "dense"
    else:
        def mv(x):
            f = ib.spread_tilde(g, prob.q, x.reshape(prob.N, d))
            v, _ = stokes_solve(g, f)
            return ib.interp(g, prob.q, v).ravel()

        op = spla.LinearOperator((prob.N * d, prob.N * d), matvec=mv, dtype=np.float64)
        it = [0]

        def cb(_):
            it[0] += 1

        lam, flag = spla.cg(op, rhs, rtol=cg_tol, atol=0.0, maxiter=cg_maxiter, callback=cb)
        info["method"] = "cg"
        info["cg_iters"] = it[0]
        info["cg_flag"] = int(flag)
    lam = lam.reshape(prob.N, d)
    f = ib.spread_tilde(g, prob.q, lam)
    f = [g_force[a] + f[a] for a in range(d)]
    v, p = stokes_solve(g, f, h_div)
    if return_info:
        return v, p, lam, info
    return v, p, lam
