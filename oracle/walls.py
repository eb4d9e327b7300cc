"""Constrained Stokes system with physical walls (App. D), FP64, test
infrastructure only.

Axes are periodic, or bounded by walls at x_a = 0 and x_a = L_a on which the
fluid velocity is given (no-slip: zero; inflow/outflow or a moving wall:
boundary data).  Field layout (the same in the GPU library, so fields compare
entry by entry): every field holds n_0 x ... x n_{d-1} values (numpy shape
n[::-1], x fastest).  Along a wall axis a, cell-centred quantities (pressure,
the velocity components tangential to the wall) have their n cell centres;
the normal component v_a lives on the faces i h, i = 0..n, of which i = 0..n-1
are stored: the stored i = 0 face lies on the low wall and is a boundary
entry (its equation is `v = wall value`), the high wall face i = n is not
stored.

Boundary treatment (App. D): a field is extended beyond the walls by an
affine map u_ext = E u + c, by linear extrapolation through the wall value:
  tangential velocity: ghost = 2 u_wall - (mirror interior value)
  normal velocity:     wall faces carry the wall value u_b; beyond the wall
                       u(-k) = 2 u_b - u(k)
  pressure:            ghost = + (mirror interior value)  (homogeneous Neumann)
and the standard operators are applied to the extended field.  The same
extension gives interpolation, J_BC u = J_0 (E u + c), and spreading,
S_BC = E^T S_0 (the adjoint for homogeneous data).  On several axes E is the
product of the one-axis extensions.

Two independent routes:
  * route K: sparse matrices assembled from 1-D operators by Kronecker sums
    (used for the solves), J from the composed one-axis extensions;
  * route X: the definition above, applied literally to ghost-extended arrays
    (used to pin route K, and to form the boundary-data terms).
A third route, `solve_dst`, solves the fluid block with exact separable
transforms of the velocity operator and a dense pressure Schur complement.

Inhomogeneous data (the c term) enters the fluid equations only; markers are
expected to stay out of the kernel support of walls that carry nonzero data
(J_0 c is not formed).
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy import fft as sfft

from .peskin import phi

PFIELD = -1  # field code of the pressure (velocity components are 0..d-1)


# ---------------------------------------------------------------- route K ---
def _lap1d(n, kind):
    """Dimensionless 1-D second difference for one axis.
    'per': periodic; 'cdir': cell-centred, ghost = -u; 'cneu': cell-centred,
    ghost = +u; 'vert': faces 0..n-1 of an axis whose faces 0 and n are walls
    (the face-0 column and row are zero: face 0 is boundary data)."""
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    M = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="lil")
    if kind == "per":
        M[0, n - 1] = 1.0
        M[n - 1, 0] = 1.0
    elif kind == "cdir":
        M[0, 0] = -3.0
        M[n - 1, n - 1] = -3.0
    elif kind == "cneu":
        M[0, 0] = -1.0
        M[n - 1, n - 1] = -1.0
    elif kind == "vert":
        M[0, :] = 0.0
        M[:, 0] = 0.0
    else:
        raise ValueError(kind)
    return M.tocsr()


def _grad1d(n, periodic):
    """Cell-to-face difference p_i - p_{i-1} on face i = 0..n-1 (wall axis:
    face 0 is a boundary face and gets no gradient)."""
    M = sp.lil_matrix((n, n))
    for i in range(n):
        if i > 0:
            M[i, i] = 1.0
            M[i, i - 1] = -1.0
        elif periodic:
            M[0, 0] = 1.0
            M[0, n - 1] = -1.0
    return M.tocsr()


def _kron(mats):
    """Kronecker product of per-axis matrices, axis 0 fastest."""
    out = sp.identity(1, format="csr")
    for M in mats[::-1]:
        out = sp.kron(out, M, format="csr")
    return out


class WallGrid:
    """n cells per axis, box L, walls[a] True for walls at both ends of axis a."""

    def __init__(self, n, L, walls, eta=1.0, rho=0.0, dt=0.0):
        self.n = tuple(int(v) for v in n)
        self.d = len(self.n)
        self.L = tuple(float(v) for v in L)
        self.walls = tuple(bool(w) for w in walls)
        self.h = self.L[0] / self.n[0]
        assert all(abs(self.L[a] / self.n[a] - self.h) < 1e-12 * self.h for a in range(self.d))
        self.eta, self.rho, self.dt = float(eta), float(rho), float(dt)
        self.shape = self.n[::-1]
        self.ncell = int(np.prod(self.n))

    @property
    def sigma(self):
        return 0.0 if (self.rho == 0.0 or self.dt == 0.0) else self.rho / self.dt

    def ax(self, a):
        """numpy axis of grid axis a"""
        return self.d - 1 - a

    def kind(self, field, a):
        if not self.walls[a]:
            return "per"
        if field == PFIELD:
            return "cneu"
        return "vert" if field == a else "cdir"

    def face_shape(self, a):
        s = list(self.shape)
        del s[self.ax(a)]
        return tuple(s)

    def boundary_mask(self, c):
        """stored wall faces of velocity component c (index 0 along its own wall axis)"""
        m = np.zeros(self.shape, dtype=bool)
        if self.walls[c]:
            idx = [slice(None)] * self.d
            idx[self.ax(c)] = 0
            m[tuple(idx)] = True
        return m

    def zero_data(self):
        return {(a, s): np.zeros((self.d,) + self.face_shape(a))
                for a in range(self.d) if self.walls[a] for s in (0, 1)}

    # -- route K matrices
    def lap_matrix(self, field):
        I = [sp.identity(m, format="csr") for m in self.n]
        total = None
        for b in range(self.d):
            ms = list(I)
            ms[b] = _lap1d(self.n[b], self.kind(field, b))
            t = _kron(ms)
            total = t if total is None else total + t
        return total

    def A_matrix(self):
        """sigma I - eta h^-2 Lap per component, identity rows on wall faces"""
        blocks = []
        for c in range(self.d):
            Ac = (self.sigma * sp.identity(self.ncell) - (self.eta / self.h ** 2) * self.lap_matrix(c)).tolil()
            for r in np.nonzero(self.boundary_mask(c).ravel())[0]:
                Ac.rows[r] = [int(r)]
                Ac.data[r] = [1.0]
            blocks.append(Ac.tocsr())
        return sp.block_diag(blocks, format="csr")

    def G_matrix(self):
        I = [sp.identity(m, format="csr") for m in self.n]
        rows = []
        for c in range(self.d):
            ms = list(I)
            ms[c] = _grad1d(self.n[c], not self.walls[c])
            rows.append(_kron(ms) / self.h)
        return sp.vstack(rows, format="csr")

    def D_matrix(self):
        return -self.G_matrix().T.tocsr()

    # -- extension (one axis), shared by the composed J of route K
    def ext_index(self, field, a, j):
        """extended index j along axis a -> [(stored index, coefficient)] of
        the homogeneous part E (the data part c is not included)."""
        n = self.n[a]
        kind = self.kind(field, a)
        if kind == "per":
            return [(j % n, 1.0)]
        if kind in ("cdir", "cneu"):
            s = -1.0 if kind == "cdir" else 1.0
            if j < 0:
                return [(-j - 1, s)]
            if j >= n:
                return [(2 * n - 1 - j, s)]
            return [(j, 1.0)]
        if j == 0 or j == n:  # wall faces: data only
            return []
        if j < 0:
            return [(-j, -1.0)]
        if j > n:
            return [(2 * n - j, -1.0)]
        return [(j, 1.0)]

    def J_matrix(self, q):
        """J_BC (homogeneous part) = J_0 E, dense (N d) x (d ncell)."""
        q = np.asarray(q, dtype=np.float64).reshape(-1, self.d)
        N, d = q.shape[0], self.d
        Jm = np.zeros((N * d, d * self.ncell))
        strides = [int(np.prod(self.n[:b])) for b in range(d)]
        for c in range(d):
            for i in range(N):
                wins = []
                for b in range(d):
                    s = q[i, b] / self.h - (0.0 if b == c else 0.5)
                    j0 = int(np.floor(s)) - 1
                    wins.append([(j0 + m, float(phi(np.array([s - (j0 + m)]))[0])) for m in range(4)])
                for combo in itertools.product(*wins):
                    w = float(np.prod([t[1] for t in combo]))
                    if w == 0.0:
                        continue
                    targets = [(0, w)]
                    for b, (j, _) in enumerate(combo):
                        ext = self.ext_index(c, b, j)
                        targets = [(t + e * strides[b], cf * ce) for (t, cf) in targets for (e, ce) in ext]
                    for t, cf in targets:
                        Jm[i * d + c, c * self.ncell + t] += cf
        return Jm

    # ------------------------------------------------------------ route X ---
    def _wall_values(self, bd, a, s, c):
        """wall data of component c on wall (a, s) broadcast to the field shape
        with the wall axis kept as length 1"""
        v = np.asarray(bd[(a, s)][c], dtype=np.float64)
        return np.expand_dims(v, self.ax(a))

    def extend1(self, u, field, bd):
        """one ghost layer on every axis (corners unused): periodic wrap, or
        E u + c on walls.  For the normal component on its own wall axis the
        stored face 0 is replaced by the wall value and face n is appended.
        Returns the extended array; index j of axis a sits at j + 1."""
        e = np.asarray(u, dtype=np.float64)
        for a in range(self.d):
            ax = self.ax(a)
            n = self.n[a]
            kind = self.kind(field, a)
            take = lambda arr, i: np.take(arr, [i], axis=ax)
            if kind == "per":
                lo, hi = take(e, n - 1), take(e, 0)
                e = np.concatenate([lo, e, hi], axis=ax)
            elif kind == "cneu":
                e = np.concatenate([take(e, 0), e, take(e, n - 1)], axis=ax)
            elif kind == "cdir":
                wl = self._ext_data(bd, a, 0, field, e.shape, ax)
                wh = self._ext_data(bd, a, 1, field, e.shape, ax)
                e = np.concatenate([2 * wl - take(e, 0), e, 2 * wh - take(e, n - 1)], axis=ax)
            else:  # vert
                ub_lo = self._ext_data(bd, a, 0, field, e.shape, ax)
                ub_hi = self._ext_data(bd, a, 1, field, e.shape, ax)
                idx = [slice(None)] * self.d
                idx[ax] = slice(1, None)
                inner = e[tuple(idx)]
                e = np.concatenate([2 * ub_lo - take(e, 1), ub_lo, inner, ub_hi], axis=ax)
        return e

    def _ext_data(self, bd, a, s, field, cur_shape, ax):
        """wall data for `field` on wall (a, s), extended over the axes
        already extended: periodically on periodic axes, by zeros on wall
        axes (those corners are read by no stencil of this module)."""
        if bd is None or field == PFIELD:
            shp = list(cur_shape)
            shp[ax] = 1
            return np.zeros(shp)
        v = self._wall_values(bd, a, s, field)
        for b in range(self.d):
            axb = self.ax(b)
            if axb != ax and v.shape[axb] != cur_shape[axb]:
                pad = [(0, 0)] * self.d
                pad[axb] = (1, cur_shape[axb] - v.shape[axb] - 1)
                v = np.pad(v, pad, mode="wrap" if not self.walls[b] else "constant")
        return v

    def apply_full(self, v, p, bd):
        """Route X: the affine fluid operator.  Returns (momentum rows per
        component, divergence rows), momentum = sigma v - eta h^-2 Lap v + G p
        (wall-face rows: the stored value), divergence = D v (not negated)."""
        d, h = self.d, self.h
        pe = self.extend1(p, PFIELD, None)
        core = tuple([slice(1, -1)] * d)
        mom = []
        div = np.zeros(self.shape)
        for c in range(d):
            ue = self.extend1(v[c], c, bd)
            ax_c = self.ax(c)
            n_c = self.n[c]
            # vertical component on a wall axis: extended along c by 3 layers
            # (ghost, wall face 0 replaced, ..., wall face n): core is 1..n
            sl = [slice(1, 1 + self.n[b]) for b in range(d)][::-1]
            lap = -2.0 * d * ue[tuple(sl)]
            for b in range(d):
                axb = self.ax(b)
                for sh in (-1, 1):
                    s2 = list(sl)
                    s2[axb] = slice(sl[axb].start + sh, sl[axb].stop + sh)
                    lap = lap + ue[tuple(s2)]
            # pressure gradient on face i_c: p_i - p_{i-1}
            s_hi = [slice(1, 1 + self.n[b]) for b in range(d)][::-1]
            s_lo = list(s_hi)
            s_lo[ax_c] = slice(0, n_c)
            gp = (pe[tuple(s_hi)] - pe[tuple(s_lo)]) / h
            m = self.sigma * ue[tuple(sl)] - (self.eta / h ** 2) * lap + gp
            bm = self.boundary_mask(c)
            m[bm] = np.asarray(v[c])[bm]
            mom.append(m)
            # divergence: face i_c + 1 minus face i_c (wall faces carry data)
            s_up = list(sl)
            s_up[ax_c] = slice(2, 2 + n_c)
            div = div + (ue[tuple(s_up)] - ue[tuple(sl)]) / h
        return mom, div

    def extend2_homog(self, u, field):
        """two ghost layers on every axis with the homogeneous extension E
        (periodic wrap, mirrors with signs); for the normal component on its
        own wall axis the wall faces hold zero and face n..n+2 are appended.
        Index j of axis a sits at j + 2."""
        assert field != PFIELD
        e = np.asarray(u, dtype=np.float64).copy()
        for a in range(self.d):
            ax = self.ax(a)
            n = self.n[a]
            kind = self.kind(field, a)
            take = lambda arr, i: np.take(arr, [i], axis=ax)
            if kind == "per":
                e = np.concatenate([take(e, n - 2), take(e, n - 1), e, take(e, 0), take(e, 1)], axis=ax)
            elif kind == "cdir":
                e = np.concatenate([-take(e, 1), -take(e, 0), e, -take(e, n - 1), -take(e, n - 2)], axis=ax)
            else:
                z = 0.0 * take(e, 0)
                idx = [slice(None)] * self.d
                idx[ax] = slice(1, None)
                inner = e[tuple(idx)]
                e = np.concatenate([-take(e, 2), -take(e, 1), z, inner, z, -take(e, n - 1), -take(e, n - 2)],
                                   axis=ax)
        return e

    def interp_bruteforce(self, v, q):
        """J_0 E v by summing the kernel over every node of the two-layer
        extended grid (no window arithmetic)."""
        q = np.asarray(q, dtype=np.float64).reshape(-1, self.d)
        out = np.zeros((q.shape[0], self.d))
        for c in range(self.d):
            ue = self.extend2_homog(v[c], c)
            coords = []
            for b in range(self.d):
                m = ue.shape[self.ax(b)]
                off = 0.0 if b == c else 0.5
                coords.append((np.arange(m) - 2 + off) * self.h)
            for i in range(q.shape[0]):
                w = np.ones(ue.shape)
                for b in range(self.d):
                    wb = phi((q[i, b] - coords[b]) / self.h)
                    shp = [1] * self.d
                    shp[self.ax(b)] = -1
                    w = w * wb.reshape(shp)
                out[i, c] = float(np.sum(w * ue))
        return out


# ------------------------------------------------------------- problem ----
class WallProblem:
    """The constrained system of Eq. constrained_Stokes with walls, unknowns
    [v_0 .. v_{d-1} | pi | Lambda]; prescribed rigid motion W = -K U is
    supplied by the caller as W (length N d)."""

    def __init__(self, wg: WallGrid, q):
        self.g = wg
        self.q = np.asarray(q, dtype=np.float64).reshape(-1, wg.d)
        self.N = self.q.shape[0]
        self.J = wg.J_matrix(self.q) if self.N else np.zeros((0, wg.d * wg.ncell))

    @property
    def size(self):
        return (self.g.d + 1) * self.g.ncell + self.g.d * self.N

    def split(self, x):
        g = self.g
        n, d = g.ncell, g.d
        v = [x[c * n:(c + 1) * n].reshape(g.shape) for c in range(d)]
        p = x[d * n:(d + 1) * n].reshape(g.shape)
        lam = x[(d + 1) * n:].reshape(-1, d)
        return v, p, lam

    def join(self, v, p, lam):
        return np.concatenate([np.concatenate([np.ravel(a) for a in v]), np.ravel(p), np.ravel(lam)])

    def matrix(self):
        g = self.g
        A = g.A_matrix()
        G = g.G_matrix()
        D = g.D_matrix()
        J = sp.csr_matrix(self.J)
        S = (J.T / g.h ** g.d).tocsr()
        if not any(g.walls) and g.sigma == 0.0:
            raise ValueError("periodic steady Stokes: use system.Problem")
        return sp.bmat([[A, G, -S], [-D, None, None], [-J, None, None]], format="csr")

    def rhs(self, W, g_force=None, bd=None):
        """b = [g + data terms (wall rows: wall value); h = data terms; W]"""
        wg = self.g
        d = wg.d
        bd = wg.zero_data() if bd is None else bd
        gf = [np.zeros(wg.shape) for _ in range(d)] if g_force is None else [np.asarray(x, float) for x in g_force]
        zero_v = [np.zeros(wg.shape) for _ in range(d)]
        mom0, div0 = wg.apply_full(zero_v, np.zeros(wg.shape), bd)
        rows = []
        for c in range(d):
            r = gf[c] - mom0[c]
            bm = wg.boundary_mask(c)
            if bm.any():
                r[bm] = np.broadcast_to(wg._wall_values(bd, c, 0, c), wg.shape)[bm]
            rows.append(r)
        hrow = div0  # -D v_int = h  with  -D_full v = 0  ->  -D v_int = D(data)
        return np.concatenate([np.concatenate([r.ravel() for r in rows]), hrow.ravel(),
                               np.asarray(W, dtype=np.float64).ravel()])

    def solve(self, b, refine=3):
        """Sparse LU of the system bordered by <pi> = 0, plus a few steps of
        iterative refinement in FP64 (removes the rounding the factorisation
        leaves; the result is the exact solution)."""
        wg = self.g
        n, d = wg.ncell, wg.d
        M = self.matrix()
        c = np.zeros(self.size)
        c[d * n:(d + 1) * n] = 1.0 / n
        B = sp.bmat([[M, sp.csr_matrix(c).T], [sp.csr_matrix(c), None]], format="csc")
        lu = spla.splu(B)
        rhs = np.concatenate([b, [0.0]])
        sol = lu.solve(rhs)
        for _ in range(refine):
            sol = sol + lu.solve(rhs - B @ sol)
        return sol[: self.size]

    def residual(self, x, b):
        return float(np.linalg.norm(b - self.matrix() @ x) / np.linalg.norm(b))


# ------------------------------------------------ independent fluid route ---
def _axis_transform(wg, c, a):
    """(forward, inverse, eigenvalues) of the 1-D Laplacian of component c on
    axis a: DFT (periodic), DST-II (cell-centred Dirichlet mirror), DST-I on
    faces 1..n-1 (normal component between walls)."""
    n = wg.n[a]
    kind = wg.kind(c, a)
    ax = wg.ax(a)
    if kind == "per":
        lam = -4.0 * np.sin(np.pi * np.arange(n) / n) ** 2
        return (lambda x: sfft.fft(x, axis=ax), lambda y: sfft.ifft(y, axis=ax), lam)
    if kind == "cdir":
        lam = -4.0 * np.sin(np.pi * np.arange(1, n + 1) / (2 * n)) ** 2
        return (lambda x: sfft.dst(x, type=2, axis=ax, norm="ortho"),
                lambda y: sfft.idst(y, type=2, axis=ax, norm="ortho"), lam)
    lam = -4.0 * np.sin(np.pi * np.arange(1, n) / (2 * n)) ** 2

    def fwd(x):
        idx = [slice(None)] * wg.d
        idx[ax] = slice(1, None)
        return sfft.dst(x[tuple(idx)], type=1, axis=ax, norm="ortho")

    def inv(y):
        z = sfft.idst(y, type=1, axis=ax, norm="ortho")
        pad = [(0, 0)] * wg.d
        pad[ax] = (1, 0)
        return np.pad(z, pad)

    return fwd, inv, lam


def apply_Ainv(wg, f, c):
    """exact A^-1 on component c by separable transforms (wall faces: identity)"""
    f = np.asarray(f, dtype=np.float64)
    tr = [_axis_transform(wg, c, a) for a in range(wg.d)]
    y = f.astype(complex) if any(wg.kind(c, a) == "per" for a in range(wg.d)) else f.copy()
    for a in range(wg.d):
        y = tr[a][0](y)
    den = np.full(y.shape, wg.sigma, dtype=np.float64)
    for a in range(wg.d):
        shp = [1] * wg.d
        shp[wg.ax(a)] = -1
        den = den - (wg.eta / wg.h ** 2) * tr[a][2].reshape(shp)
    y = y / den
    for a in reversed(range(wg.d)):
        y = tr[a][1](y)
    u = np.real(y)
    bm = wg.boundary_mask(c)
    u[bm] = f[bm]
    return u


def stokes_solve_dst(wg, g_rows, h_rows):
    """Solves [A G; -D 0][v; p] = [g; h] with <p> = 0 by exact A^-1 (separable
    transforms) and a dense pressure Schur complement D A^-1 G."""
    d, n = wg.d, wg.ncell
    G = wg.G_matrix().toarray()
    D = -G.T
    Ainv = lambda vec: np.concatenate([apply_Ainv(wg, vec[c * n:(c + 1) * n].reshape(wg.shape), c).ravel()
                                       for c in range(d)])
    AinvG = np.stack([Ainv(G[:, k]) for k in range(n)], axis=1)
    Sp = D @ AinvG
    gv = np.concatenate([np.ravel(x) for x in g_rows])
    rhs = D @ Ainv(gv) + np.ravel(h_rows)
    # -D v = h, v = A^-1 (g - G p)  ->  D A^-1 G p = D A^-1 g + h
    B = np.block([[Sp, np.ones((n, 1)) / n], [np.ones((1, n)) / n, np.zeros((1, 1))]])
    p = np.linalg.solve(B, np.concatenate([rhs, [0.0]]))[:n]
    v = Ainv(gv - G @ p)
    return [v[c * n:(c + 1) * n].reshape(wg.shape) for c in range(d)], p.reshape(wg.shape)


def solve_schur_dst(prob: WallProblem, b):
    """The whole system by the Schur route of Sec. V.A with exact fluid solves:
    M = J L^-1 S (dense, column by column), M Lambda = -(W + J v~),
    v = v~ + L^-1 S Lambda."""
    wg = prob.g
    d, n = wg.d, wg.ncell
    gb = [b[c * n:(c + 1) * n].reshape(wg.shape) for c in range(d)]
    hb = b[d * n:(d + 1) * n].reshape(wg.shape)
    W = b[(d + 1) * n:]
    vt, pt = stokes_solve_dst(wg, gb, hb)
    J = prob.J
    S = J.T / wg.h ** d
    cols = []
    for k in range(J.shape[0]):
        sv, _ = stokes_solve_dst(wg, [S[c * n:(c + 1) * n, k].reshape(wg.shape) for c in range(d)],
                                 np.zeros(wg.shape))
        cols.append(J @ np.concatenate([x.ravel() for x in sv]))
    M = np.stack(cols, axis=1)
    lam = np.linalg.solve(M, -(W + J @ np.concatenate([x.ravel() for x in vt])))
    sv, sp_ = stokes_solve_dst(wg, [(S @ lam)[c * n:(c + 1) * n].reshape(wg.shape) for c in range(d)],
                               np.zeros(wg.shape))
    v = [vt[c] + sv[c] for c in range(d)]
    p = pt + sp_
    return prob.join(v, p, lam)
