"""Free kinematics: bodies under a given force and torque (Sec. II) whose rigid
velocities are unknowns (Sec. VIII: the body mobility N = (K* M^-1 K)^-1).

The enlarged system is referred to in the paper but its display is elided
in the source; it is read here as the constrained system of ``system`` with
the rigid velocities U_f of the free bodies added as unknowns and force balance
added as equations:

  [ A   G  -S~   0   ] [v     ]   [g]
  [-D   0   0    0   ] [pi    ] = [0]
  [-J   0   0    K_f ] [Lambda]   [W]     W_i = -(K U)_i on prescribed bodies'
  [ 0   0   K_f^T 0  ] [U_f   ]   [F]     markers, 0 on free bodies' markers

Row 3 makes each free body's markers move rigidly with U_f; row 4 says the
force and torque the body exerts on the fluid, K_f^T Lambda, equal the applied
load F (no inertia).  Eliminating the fluid gives M Lambda - K_f U_f = -(W + J v~)
and K_f^T Lambda = F, i.e. U_f = N (F - K_f^T M^-1 (-(W + J v~)))-type relations
with N^-1 = K_f^T M^-1 K_f, the resistance matrix.

Vector layout: [v | pi | Lambda | U_f], U_f body-major over the free bodies
(in body order), each (d + rot) long.
"""
import numpy as np

from . import fft_stokes, ib
from .system import Problem


class FreeProblem:
    def __init__(self, prob: Problem, free):
        self.p = prob
        self.free = np.asarray(free, dtype=bool).reshape(prob.nbody)
        self.fidx = np.nonzero(self.free)[0]
        d = prob.grid.d
        self.nr = d + (1 if d == 2 else 3)
        self.nU = len(self.fidx) * self.nr
        # K_f: dN x nU, columns = rigid modes of the free bodies
        Kf = np.zeros((prob.N * d, self.nU))
        for fb, b in enumerate(self.fidx):
            for c in range(self.nr):
                UO = np.zeros((prob.nbody, self.nr))
                UO[b, c] = 1.0
                V = ib.apply_K(prob.rel, prob.body, UO, d)
                V[prob.body != b] = 0.0
                Kf[:, fb * self.nr + c] = V.ravel()
        self.Kf = Kf

    @property
    def size(self):
        return self.p.size + self.nU

    def split(self, x):
        v, p, lam = self.p.split(x[: self.p.size])
        return v, p, lam, x[self.p.size:]

    def join(self, v, p, lam, U):
        return np.concatenate([self.p.join(v, p, lam), np.asarray(U, dtype=np.float64).ravel()])

    def rhs(self, UO_all, g_force=None):
        """UO_all[b] = (U, Omega) of a prescribed body b, (F, T) of a free one."""
        pr = self.p
        d = pr.grid.d
        UO_all = np.asarray(UO_all, dtype=np.float64).reshape(pr.nbody, self.nr)
        UOp = UO_all.copy()
        UOp[self.free] = 0.0
        b = pr.rhs(UOp, g_force)  # W = -K U_prescribed; zero on free bodies' markers
        F = UO_all[self.free].ravel()
        return np.concatenate([b, F])

    def matvec(self, x):
        pr = self.p
        y = pr.matvec(x[: pr.size])
        U = x[pr.size:]
        lam = x[pr.size - pr.N * pr.grid.d: pr.size]
        y[pr.size - pr.N * pr.grid.d:] += self.Kf @ U
        return np.concatenate([y, self.Kf.T @ lam])

    def residual(self, x, b):
        return float(np.linalg.norm(b - self.matvec(x)) / np.linalg.norm(b))

    def solve_dense(self, b):
        """Bordered LU of the enlarged system (tiny grids)."""
        pr = self.p
        M = pr.dense_matrix()
        n0 = pr.size
        nL = pr.N * pr.grid.d
        Mf = np.zeros((self.size, self.size))
        Mf[:n0, :n0] = M
        Mf[n0 - nL:n0, n0:] = self.Kf
        Mf[n0:, n0 - nL:n0] = self.Kf.T
        C = pr.constraint_rows()
        C = np.hstack([C, np.zeros((C.shape[0], self.nU))])
        k = C.shape[0]
        Bd = np.zeros((self.size + k, self.size + k))
        Bd[: self.size, : self.size] = Mf
        Bd[: self.size, self.size:] = C.T
        Bd[self.size:, : self.size] = C
        sol = np.linalg.solve(Bd, np.concatenate([b, np.zeros(k)]))
        return sol[: self.size]


def solve_free_fft(fp: FreeProblem, UO_all, g_force=None):
    """Exact solution by the Schur route: with the true mobility M = J L^-1 S~,
      [ M    -K_f ] [Lambda]   [-(W + J v~)]
      [ K_f^T  0  ] [U_f   ] = [ F         ]
    then v = L^-1 (g + S~ Lambda) (periodic DFT solves)."""
    pr = fp.p
    g = pr.grid
    d = g.d
    if g_force is None:
        g_force = [np.zeros(g.shape) for _ in range(d)]
    UO_all = np.asarray(UO_all, dtype=np.float64).reshape(pr.nbody, fp.nr)
    UOp = UO_all.copy()
    UOp[fp.free] = 0.0
    W = -ib.apply_K(pr.rel, pr.body, UOp, d)
    vt, _ = fft_stokes.stokes_solve(g, g_force)
    r1 = -(W + ib.interp(g, pr.q, vt)).ravel()
    M = fft_stokes.mobility_true(pr)
    nL = pr.N * d
    Bm = np.zeros((nL + fp.nU, nL + fp.nU))
    Bm[:nL, :nL] = M
    Bm[:nL, nL:] = -fp.Kf
    Bm[nL:, :nL] = fp.Kf.T
    sol = np.linalg.solve(Bm, np.concatenate([r1, UO_all[fp.free].ravel()]))
    lam = sol[:nL].reshape(pr.N, d)
    U = sol[nL:]
    f = ib.spread_tilde(g, pr.q, lam)
    v, p = fft_stokes.stokes_solve(g, [g_force[a] + f[a] for a in range(d)])
    return v, p, lam, U


def resistance(fp: FreeProblem):
    """R = K_f^T M^-1 K_f (the inverse of the free bodies' mobility N)."""
    M = fft_stokes.mobility_true(fp.p)
    return fp.Kf.T @ np.linalg.solve(M, fp.Kf)
