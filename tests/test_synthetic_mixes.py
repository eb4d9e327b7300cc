"""The seeded problem mixes of the batch (config 4) and the serving stream
(config 5) follow their stated recipes (CPU only): grid sizes from the given
sets, body counts and sizes in range, bounding shapes at least 4h apart in
the periodic box, markers at the stated spacing, Poisson arrivals at the
given rate, and the same seed giving the same mix."""
import numpy as np
import pytest

from oracle.ib import quat_rotate
from synthetic import batch_2d, ellipsoid_markers, random_quaternion, serve_3d
from synthetic.workloads import _periodic_gap

pytest.importorskip("scipy")
from scipy.spatial import cKDTree  # noqa: E402


def test_batch_2d_recipe():
    reqs = batch_2d(64)
    assert len(reqs) == 64
    for r in reqs:
        n = r.n[0]
        assert r.n == (n, n) and n in (64, 128, 256, 512)
        h = 1.0 / n
        assert 1 <= len(r.rels) <= 8 and r.UO.shape == (len(r.rels), 3)
        radii = [s[1] for s in r.shapes]
        assert all(0.05 <= a <= 0.15 for a in radii)
        for i in range(len(radii)):
            for j in range(i + 1, len(radii)):
                assert _periodic_gap(r.centers[i], r.centers[j]) >= radii[i] + radii[j] + 4 * h - 1e-12
        for rel, a in zip(r.rels, radii):
            assert np.allclose(np.hypot(rel[:, 0], rel[:, 1]), a)
            d = np.hypot(*np.diff(np.vstack([rel, rel[:1]]), axis=0).T)
            assert abs(d.mean() / h - 2.0) < 0.15  # arc spacing ~2h
    again = batch_2d(64)
    assert all(np.array_equal(a.UO, b.UO) and a.n == b.n for a, b in zip(reqs, again))


def test_serve_3d_recipe_and_arrivals():
    reqs = serve_3d(200, rate=50.0)
    t = np.array([r.t_arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps of mean 1/50 s: the sample mean within 4 standard errors
    assert abs(gaps.mean() - 0.02) < 4 * 0.02 / np.sqrt(len(gaps))
    assert {r.n[0] for r in reqs} <= {64, 96, 128, 192}
    for r in reqs[:12]:
        h = 1.0 / r.n[0]
        assert 1 <= len(r.rels) <= 16 and r.UO.shape == (len(r.rels), 6)
        bound = [s[1] * s[2] for s in r.shapes]
        for (kind, b, asp) in r.shapes:
            assert 0.05 <= b <= 0.12 and 1.0 <= asp <= 3.0
            assert (kind == "sphere") == (asp == 1.0)
        for i in range(len(bound)):
            for j in range(i + 1, len(bound)):
                assert _periodic_gap(r.centers[i], r.centers[j]) >= bound[i] + bound[j] + 4 * h - 1e-12


@pytest.mark.parametrize("b,aspect,n", [(0.05, 1.0, 64), (0.08, 2.5, 96), (0.12, 3.0, 128)])
def test_ellipsoid_markers_on_surface_at_spacing(b, aspect, n):
    h = 1.0 / n
    pts = ellipsoid_markers(b, aspect, h)
    a = aspect * b
    # on the surface x^2/a^2 + (y^2 + z^2)/b^2 = 1
    assert np.allclose(pts[:, 0] ** 2 / a ** 2 + (pts[:, 1] ** 2 + pts[:, 2] ** 2) / b ** 2, 1.0)
    dist, _ = cKDTree(pts).query(pts, k=2)
    assert dist[:, 1].max() <= 2.2 * h + 1e-12


def test_random_quaternions_are_rotations():
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = random_quaternion(rng)
        assert abs(np.linalg.norm(q) - 1.0) < 1e-12
        R = quat_rotate(q, np.eye(3)).T  # columns: the images of e_x, e_y, e_z
        assert np.allclose(R @ R.T, np.eye(3)) and abs(np.linalg.det(R) - 1.0) < 1e-12
