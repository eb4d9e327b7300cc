"""The rigidly constrained Stokes saddle-point system (Sec. III.B-D).

Unknown x = [v; pi; Lambda], right-hand side b = [g; h; W]:

  [ A   G  -S~ ] [v     ]   [g]
  [-D   0   0  ] [pi    ] = [h]          Eq. constrained_Stokes, with
  [-J   0   0  ] [Lambda]   [W]          S~ = S - vol^-1 1^T for periodic
                                         steady Stokes (Eq. constrained_periodic)

Periodic steady Stokes adds <v> = 0 (the d mean velocities) and the pressure
is fixed by <pi> = 0; for finite rho/dt only <pi> = 0 is needed (Sec. III.D).

Flat vector layout: v^0 | ... | v^{d-1} | pi | Lambda (marker-major, i*d+alpha),
each grid block in the numpy layout of ``Grid.shape``.
"""
import numpy as np

from . import ib
from .mac import flat, unflat


class Problem:
    """Grid + markers of one or more rigid bodies (prescribed kinematics)."""

    def __init__(self, grid, q, rel, body, nbody):
        self.grid = grid
        self.q = np.asarray(q, dtype=np.float64).reshape(-1, grid.d)
        self.rel = np.asarray(rel, dtype=np.float64).reshape(-1, grid.d)
        self.body = np.asarray(body, dtype=np.int64)
        self.nbody = int(nbody)
        self.N = self.q.shape[0]

    @property
    def size(self):
        g = self.grid
        return (g.d + 1) * g.ncell + g.d * self.N

    def split(self, x):
        g = self.grid
        n = g.ncell
        v = unflat(g, x[: g.d * n], g.d)
        p = x[g.d * n:(g.d + 1) * n].reshape(g.shape)
        lam = x[(g.d + 1) * n:].reshape(self.N, g.d)
        return v, p, lam

    def join(self, v, p, lam):
        return np.concatenate([flat(v), np.asarray(p).ravel(), np.asarray(lam).ravel()])

    def matvec(self, x):
        """y = (system matrix) x, matrix-free."""
        g = self.grid
        v, p, lam = self.split(x)
        Av = g.apply_A(v)
        Gp = g.grad(p)
        Sl = ib.spread_tilde(g, self.q, lam)
        rv = [Av[a] + Gp[a] - Sl[a] for a in range(g.d)]
        rp = -g.div(v)
        rl = -ib.interp(g, self.q, v)
        return self.join(rv, rp, rl)

    def rhs(self, UO, g_force=None, h_div=None):
        """b = [g; h; W] with W = -K U (the no-slip constraint J v = K U)."""
        gr = self.grid
        if g_force is None:
            g_force = [np.zeros(gr.shape) for _ in range(gr.d)]
        if h_div is None:
            h_div = np.zeros(gr.shape)
        W = -ib.apply_K(self.rel, self.body, UO, gr.d)
        return self.join(g_force, h_div, W)

    def residual(self, x, b):
        r = b - self.matvec(x)
        return float(np.linalg.norm(r) / np.linalg.norm(b))

    # ---- dense assembly (tiny grids) --------------------------------------
    def dense_matrix(self):
        """Assemble the system matrix from the explicit sparse G, A and the
        explicit J (not from the matrix-free routines)."""
        g = self.grid
        n = g.ncell
        d = g.d
        nv = d * n
        Gm = g.G_matrix().toarray()
        Am = g.A_matrix().toarray()
        Dm = -Gm.T
        Jm = ib.J_matrix(g, self.q)
        Sm = Jm.T / g.h ** d
        if g.steady:
            # S~ = S - vol^-1 1^T: each marker's alpha force leaves a uniform
            # density on component alpha
            for a in range(d):
                Sm[a * n:(a + 1) * n, a::d] -= 1.0 / g.vol
        M = np.zeros((self.size, self.size))
        M[:nv, :nv] = Am
        M[:nv, nv:nv + n] = Gm
        M[:nv, nv + n:] = -Sm
        M[nv:nv + n, :nv] = -Dm
        M[nv + n:, :nv] = -Jm
        return M

    def constraint_rows(self):
        """Rows of the mean constraints: <v^alpha> = 0 (steady periodic) and
        <pi> = 0."""
        g = self.grid
        n = g.ncell
        rows = []
        if g.steady:
            for a in range(g.d):
                r = np.zeros(self.size)
                r[a * n:(a + 1) * n] = 1.0 / n
                rows.append(r)
        r = np.zeros(self.size)
        r[g.d * n:(g.d + 1) * n] = 1.0 / n
        rows.append(r)
        return np.array(rows)

    def solve_dense(self, b):
        """Bordered LU solve: [[M, C^T], [C, 0]] [x; mu] = [b; 0].

        C holds the mean constraints; C^T spans the left null space of M
        (momentum means and the divergence sum vanish identically), so for a
        consistent b the multipliers mu are zero and x solves M x = b."""
        M = self.dense_matrix()
        C = self.constraint_rows()
        k = C.shape[0]
        Bd = np.zeros((self.size + k, self.size + k))
        Bd[: self.size, : self.size] = M
        Bd[: self.size, self.size:] = C.T
        Bd[self.size:, : self.size] = C
        rhs = np.concatenate([b, np.zeros(k)])
        sol = np.linalg.solve(Bd, rhs)
        return sol[: self.size], sol[self.size:]


def drag(prob, lam):
    """Force and torque of each body on the fluid, K^T Lambda; the drag on the
    body is its negative (Sec. VII.E)."""
    return ib.apply_KT(prob.rel, prob.body, lam, prob.grid.d, prob.nbody)
