"""The time-step right-hand side of the nozzle flow (Sec. VII.F), FP64, test
infrastructure only.

Each step solves the constrained system (Eq. constrained_Stokes) with the
backward-Euler viscous operator A = rho/dt I - eta h^-2 Lap and the
explicit momentum forcing

    g = (rho/dt) v^n - rho (3/2 N(v^n) - 1/2 N(v^{n-1}))   (AB2; the first
                                                           step uses N(v^0))

where N(v) = div(v v) is the centred second-order flux form on the MAC grid:
for component a at its face,

    N_a = sum_b [F_ab(+1/2) - F_ab(-1/2)] / h,
    F_aa at the cell centres between a-faces: ((v_a(i) + v_a(i+1)) / 2)^2,
    F_ab (b != a) at the edges between a-faces and b-faces:
        (v_a averaged along b) * (v_b averaged along a),

with the values beyond walls taken from the same App. D extension as the
fluid operators (walls.WallGrid.extend1, boundary data included).  Wall-face
rows carry no advection (their equation is the wall value).  The paper
cites a higher-order upwind scheme for this term; the centred flux form is
the second-order scheme used here (it conserves discrete momentum and, for
a discretely divergence-free field in a periodic box, kinetic energy).

The march stops when ||v^{n+1} - v^n|| <= tol ||v^{n+1}|| (steady state).
"""
import numpy as np


def _shift(E, wg, shifts):
    """interior window of an extended array (index j at j + 1) shifted by
    shifts {axis: offset}"""
    sl = []
    for ax_np in range(wg.d):
        a = wg.d - 1 - ax_np
        o = shifts.get(a, 0)
        sl.append(slice(1 + o, 1 + o + wg.n[a]))
    return E[tuple(sl)]


def advect(wg, v, bd=None):
    """N(v) per component (list of arrays in the field layout)."""
    d, h = wg.d, wg.h
    bd = wg.zero_data() if bd is None else bd
    E = [wg.extend1(v[c], c, bd) for c in range(d)]
    out = []
    for a in range(d):
        Na = np.zeros(wg.shape)
        for b in range(d):
            if b == a:
                fp = (0.5 * (_shift(E[a], wg, {}) + _shift(E[a], wg, {a: 1}))) ** 2
                fm = (0.5 * (_shift(E[a], wg, {a: -1}) + _shift(E[a], wg, {}))) ** 2
            else:
                ua_p = 0.5 * (_shift(E[a], wg, {}) + _shift(E[a], wg, {b: 1}))
                vb_p = 0.5 * (_shift(E[b], wg, {a: -1, b: 1}) + _shift(E[b], wg, {b: 1}))
                ua_m = 0.5 * (_shift(E[a], wg, {b: -1}) + _shift(E[a], wg, {}))
                vb_m = 0.5 * (_shift(E[b], wg, {a: -1}) + _shift(E[b], wg, {}))
                fp, fm = ua_p * vb_p, ua_m * vb_m
            Na = Na + (fp - fm) / h
        Na[wg.boundary_mask(a)] = 0.0
        out.append(Na)
    return out


def step_force(wg, v_n, N_n, N_prev):
    """g of one step (list per component)"""
    if N_prev is None:
        N_prev = N_n
    return [wg.sigma * v_n[c] - wg.rho * (1.5 * N_n[c] - 0.5 * N_prev[c]) for c in range(wg.d)]


def march(prob, W, bd, v0, nsteps, tol=0.0, force=None):
    """Backward-Euler / AB2 steps of the constrained problem `prob`
    (walls.WallProblem with rho, dt > 0) from velocity v0 (list per
    component; beyond walls the extension uses the wall values), with an
    optional constant body force added to g.  Returns (states [x after each
    step], changes [||dv|| / ||v||])."""
    wg = prob.g
    assert wg.sigma > 0.0
    v = [np.array(c, dtype=np.float64) for c in v0]
    N_prev = None
    states, changes = [], []
    for _ in range(nsteps):
        N_n = advect(wg, v, bd)
        g = step_force(wg, v, N_n, N_prev)
        if force is not None:
            g = [g[c] + force[c] for c in range(wg.d)]
        x = prob.solve(prob.rhs(W, g_force=g, bd=bd))
        vn, _, _ = prob.split(x)
        num = np.sqrt(sum(np.sum((vn[c] - v[c]) ** 2) for c in range(wg.d)))
        den = np.sqrt(sum(np.sum(vn[c] ** 2) for c in range(wg.d)))
        changes.append(num / den if den > 0 else 0.0)
        states.append(x)
        N_prev = N_n
        v = [np.array(c) for c in vn]
        if tol > 0.0 and changes[-1] <= tol:
            break
    return states, changes
