"""Staggered (MAC) grid operators on a periodic box (Sec. III, Sec. III.B).

Layout (shared by every oracle module): a cell-centred scalar on an
n_0 x ... x n_{d-1} grid is a float64 array of shape ``n[::-1]`` (x index
fastest, i.e. numpy axis d-1 is x).  Velocity component alpha lives on the
faces normal to axis alpha: entry i of component alpha is the face at
position (i + 1/2 - e_alpha/2) h, i.e. the lower face of cell i.  A velocity
field is a list of d such arrays.

Operators (Sec. III.B, Eq. constrained_Stokes and Eq. A_def):
  (G p)^alpha_i = (p_i - p_{i - e_alpha}) / h
  (D v)_i      = sum_alpha (v^alpha_{i + e_alpha} - v^alpha_i) / h,  D = -G^T
  (Lap u)_i    = sum_beta (u_{i+e_beta} + u_{i-e_beta}) - 2 d u_i   (dimensionless)
  A v          = (rho/dt) v - eta h^-2 Lap v  = eta h^-2 (beta^-1 I - Lap) v
with beta = (eta/rho) dt / h^2; rho == 0 or dt == 0 means steady Stokes.
"""
import numpy as np
import scipy.sparse as sp


class Grid:
    """Uniform periodic MAC grid: d in {2, 3}, n = cells per axis (x first)."""

    def __init__(self, n, L=None, eta=1.0, rho=0.0, dt=0.0, kernel="peskin4"):
        assert kernel in ("peskin4", "bkp6")
        self.kernel = kernel  # regularised delta of J and S (Sec. III.A)
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        assert self.d in (2, 3)
        if L is None:
            L = [1.0] * self.d
        self.L = tuple(float(v) for v in L)
        hs = [self.L[a] / self.n[a] for a in range(self.d)]
        assert max(hs) - min(hs) <= 1e-12 * max(hs), "cells must be cubes"
        self.h = hs[0]
        self.eta = float(eta)
        self.rho = float(rho)
        self.dt = float(dt)
        self.shape = self.n[::-1]
        self.ncell = int(np.prod(self.n))
        self.vol = float(np.prod(self.L))

    @property
    def steady(self):
        return self.rho == 0.0 or self.dt == 0.0

    @property
    def sigma(self):
        """Coefficient rho/dt of the identity in A (0 for steady Stokes)."""
        return 0.0 if self.steady else self.rho / self.dt

    def ax(self, alpha):
        """numpy axis of coordinate direction alpha."""
        return self.d - 1 - alpha

    # ---- matrix-free operators -------------------------------------------
    def grad(self, p):
        return [(p - np.roll(p, 1, axis=self.ax(a))) / self.h for a in range(self.d)]

    def div(self, v):
        out = np.zeros(self.shape)
        for a in range(self.d):
            out += (np.roll(v[a], -1, axis=self.ax(a)) - v[a]) / self.h
        return out

    def lap(self, u):
        out = -2.0 * self.d * u
        for b in range(self.d):
            out = out + np.roll(u, 1, axis=self.ax(b)) + np.roll(u, -1, axis=self.ax(b))
        return out

    def apply_A(self, v):
        c = self.eta / self.h ** 2
        return [self.sigma * v[a] - c * self.lap(v[a]) for a in range(self.d)]

    # ---- geometry ---------------------------------------------------------
    def face_coords(self, alpha):
        """Physical coordinates (list of d arrays, shape self.shape) of the
        faces of component alpha."""
        grids = np.meshgrid(*[np.arange(self.n[b]) for b in range(self.d)], indexing="ij")
        out = []
        for b in range(self.d):
            off = 0.0 if b == alpha else 0.5
            # meshgrid 'ij' gives shape n (x first); transpose to numpy layout
            out.append(((grids[b] + off) * self.h).T.copy())
        return out

    # ---- explicit sparse assembly (independent of the roll-based forms) ----
    def _lin(self, idx):
        """Flat index of a multi-index (x first) in numpy C order of shape n[::-1]."""
        flat = 0
        stride = 1
        for a in range(self.d):
            flat = flat + (idx[a] % self.n[a]) * stride
            stride *= self.n[a]
        return flat

    def _all_idx(self):
        g = np.meshgrid(*[np.arange(self.n[a]) for a in range(self.d)], indexing="ij")
        return [x.ravel() for x in g]

    def G_matrix(self):
        """G as a sparse (d*ncell) x ncell matrix, velocity blocks stacked by
        component, each block in the flat layout of ``self.shape``."""
        idx = self._all_idx()
        row_blocks = []
        for a in range(self.d):
            me = self._lin(idx)
            lo = list(idx)
            lo[a] = idx[a] - 1
            lo = self._lin(lo)
            n = self.ncell
            rows = np.concatenate([me, me])
            cols = np.concatenate([me, lo])
            vals = np.concatenate([np.full(me.size, 1.0 / self.h), np.full(me.size, -1.0 / self.h)])
            row_blocks.append(sp.csr_matrix((vals, (rows, cols)), shape=(n, n)))
        return sp.vstack(row_blocks).tocsr()

    def lap_matrix(self):
        """Dimensionless scalar Laplacian (2d+1 point, periodic), sparse n x n."""
        idx = self._all_idx()
        me = self._lin(idx)
        rows = [me]
        cols = [me]
        vals = [np.full(me.size, -2.0 * self.d)]
        for b in range(self.d):
            for s in (-1, 1):
                nb = list(idx)
                nb[b] = idx[b] + s
                rows.append(me)
                cols.append(self._lin(nb))
                vals.append(np.ones(me.size))
        return sp.csr_matrix(
            (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
            shape=(self.ncell, self.ncell),
        )

    def A_matrix(self):
        Ls = self.lap_matrix()
        blk = self.sigma * sp.identity(self.ncell) - (self.eta / self.h ** 2) * Ls
        return sp.block_diag([blk] * self.d).tocsr()


def flat(fields):
    """Concatenate a list of grid arrays into one flat vector."""
    return np.concatenate([np.asarray(f).ravel() for f in fields])


def unflat(grid, vec, ncomp):
    """Split a flat vector into ``ncomp`` arrays of ``grid.shape``."""
    n = grid.ncell
    return [vec[c * n:(c + 1) * n].reshape(grid.shape) for c in range(ncomp)]
