"""Pins for the oracle's interpolation, spreading and rigid-body map (CPU)."""
import numpy as np
import pytest

from oracle import ib
from oracle.mac import Grid, flat


def _markers(g, N, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 1, (N, g.d)) * np.array(g.L)


@pytest.mark.parametrize("n", [(8, 8), (6, 5, 7)])
def test_adjointness_J_equals_hd_S_transpose(n):
    # <J v, L> = h^d <v, S L>  (Sec. III.A)
    g = Grid(n, [v / n[0] for v in n])
    rng = np.random.default_rng(4)
    q = _markers(g, 7, 5)
    v = [rng.standard_normal(g.shape) for _ in range(g.d)]
    lam = rng.standard_normal((7, g.d))
    lhs = np.sum(ib.interp(g, q, v) * lam)
    rhs = g.h ** g.d * np.dot(flat(v), flat(ib.spread(g, q, lam)))
    assert lhs == pytest.approx(rhs, rel=1e-13)


@pytest.mark.parametrize("n", [(8, 8), (5, 6, 7)])
def test_window_interp_equals_bruteforce_sum(n):
    g = Grid(n, [v / n[0] for v in n])
    rng = np.random.default_rng(6)
    q = _markers(g, 5, 7)
    v = [rng.standard_normal(g.shape) for _ in range(g.d)]
    assert np.allclose(ib.interp(g, q, v), ib.interp_bruteforce(g, q, v), atol=1e-13)


def test_partition_of_unity_and_linear_reproduction():
    g = Grid((16, 16))
    q = np.array([[0.43, 0.51], [0.52, 0.37], [0.61, 0.66]])
    const = [np.full(g.shape, 3.0), np.full(g.shape, -2.0)]
    assert np.allclose(ib.interp(g, q, const), [[3.0, -2.0]] * 3, atol=1e-14)
    # first-moment condition: a linear field away from the periodic seam is
    # interpolated exactly
    X = g.face_coords(0)
    Y = g.face_coords(1)
    lin = [2.0 * X[0] - 1.0 * X[1], 0.5 * Y[0] + 3.0 * Y[1]]
    out = ib.interp(g, q, lin)
    ref = np.stack([2 * q[:, 0] - q[:, 1], 0.5 * q[:, 0] + 3 * q[:, 1]], axis=1)
    assert np.allclose(out, ref, atol=1e-13)


def test_spread_total_force_and_tilde_mean():
    g = Grid((8, 8, 8))
    q = _markers(g, 6, 8)
    lam = np.random.default_rng(9).standard_normal((6, 3))
    f = ib.spread(g, q, lam)
    for a in range(3):
        # integral of the force density = total marker force
        assert np.sum(f[a]) * g.h ** 3 == pytest.approx(lam[:, a].sum(), rel=1e-12, abs=1e-12)
        ft = ib.spread_tilde(g, q, lam)[a]
        assert abs(ft.mean()) < 1e-12


def test_K_KT_adjoint_and_rigid_motion():
    rng = np.random.default_rng(10)
    for d in (2, 3):
        rot = 1 if d == 2 else 3
        N, B = 9, 2
        rel = rng.standard_normal((N, d))
        body = np.array([0] * 5 + [1] * 4)
        UO = rng.standard_normal((B, d + rot))
        lam = rng.standard_normal((N, d))
        V = ib.apply_K(rel, body, UO, d)
        FT = ib.apply_KT(rel, body, lam, d, B)
        assert np.sum(V * lam) == pytest.approx(np.sum(UO * FT), rel=1e-13)
        # pure rotation: velocity orthogonal to the lever arm, |V| = |Omega||r| (2-D)
        UO2 = np.zeros((B, d + rot))
        UO2[:, d:] = rng.standard_normal((B, rot))
        V2 = ib.apply_K(rel, body, UO2, d)
        assert np.allclose(np.sum(V2 * rel, axis=1), 0.0, atol=1e-13)
        if d == 2:
            assert np.allclose(np.linalg.norm(V2, axis=1),
                               np.abs(UO2[body, 2]) * np.linalg.norm(rel, axis=1), rtol=1e-13)


def test_J_matrix_matches_matrix_free():
    g = Grid((6, 6))
    q = _markers(g, 4, 12)
    rng = np.random.default_rng(13)
    v = [rng.standard_normal(g.shape) for _ in range(2)]
    Jm = ib.J_matrix(g, q)
    assert np.allclose(Jm @ flat(v), ib.interp(g, q, v).ravel(), atol=1e-13)


def test_K_rotation_direction_closed_form():
    # Omega x r with the right-hand rule (Sec. II): a counter-clockwise spin
    # omega = 1 moves the lever arm (r, 0) along +y, and a spin about +z moves
    # +x towards +y; K^T gives the matching torque r x F
    r = 0.3
    V = ib.apply_K(np.array([[r, 0.0], [0.0, r]]), np.array([0, 0]), np.array([[0.0, 0.0, 1.0]]), 2)
    assert np.allclose(V, [[0.0, r], [-r, 0.0]], atol=1e-15)
    V3 = ib.apply_K(np.eye(3), np.zeros(3, dtype=np.int64), np.array([[0, 0, 0, 0.0, 0.0, 2.0]]), 3)
    assert np.allclose(V3, [[0.0, 2.0, 0.0], [-2.0, 0.0, 0.0], [0.0, 0.0, 0.0]], atol=1e-15)
    V3 = ib.apply_K(np.eye(3), np.zeros(3, dtype=np.int64), np.array([[0, 0, 0, 1.0, 0.0, 0.0]]), 3)
    assert np.allclose(V3, [[0.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]], atol=1e-15)
    # a force +y at the lever arm +x turns the body counter-clockwise
    FT = ib.apply_KT(np.array([[r, 0.0]]), np.array([0]), np.array([[0.0, 5.0]]), 2, 1)
    assert np.allclose(FT, [[0.0, 5.0, 5.0 * r]], atol=1e-15)
    FT3 = ib.apply_KT(np.array([[1.0, 0.0, 0.0]]), np.array([0]), np.array([[0.0, 0.0, 2.0]]), 3, 1)
    assert np.allclose(FT3, [[0.0, 0.0, 2.0, 0.0, -2.0, 0.0]], atol=1e-15)


def test_quaternion_rotation_hand_computed():
    s = np.sqrt(0.5)
    # 90 degrees about z: x -> y, y -> -x, z fixed
    out = ib.quat_rotate([s, 0.0, 0.0, s], np.eye(3))
    assert np.allclose(out, [[0, 1, 0], [-1, 0, 0], [0, 0, 1]], atol=1e-15)
    # 90 degrees about x: y -> z, z -> -y
    out = ib.quat_rotate([s, s, 0.0, 0.0], np.eye(3))
    assert np.allclose(out, [[1, 0, 0], [0, 0, 1], [0, -1, 0]], atol=1e-15)
    # 120 degrees about (1,1,1)/sqrt(3) cycles the axes: x -> y -> z -> x
    c, t = np.cos(np.pi / 3), np.sin(np.pi / 3) / np.sqrt(3.0)
    out = ib.quat_rotate([c, t, t, t], np.eye(3))
    assert np.allclose(out, [[0, 1, 0], [0, 0, 1], [1, 0, 0]], atol=1e-15)
    # 180 degrees about y: x -> -x; an unnormalised quaternion is normalised
    out = ib.quat_rotate([0.0, 0.0, 3.0, 0.0], np.array([[1.0, 2.0, 3.0]]))
    assert np.allclose(out, [[-1.0, 2.0, -3.0]], atol=1e-15)
