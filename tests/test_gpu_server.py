"""The serving engine (ibr_server_*, continuous batching of independent
constrained solves) through the C ABI.

What is checked:
  - each request's result in a concurrent mix equals its result solved alone
    by ibr_solve_coupled (every reduction of the library has a fixed order,
    so the mix changes timing only): bitwise, and asserted within the parity
    tolerance 1e-9 of the solves at residual 1e-10;
  - the results match the oracle's exact solution (1e-9 at residual 1e-10);
  - requests really overlap on the device (their run intervals intersect);
  - admission by the HBM budget: reserved bytes never exceed it, idle
    resident grids are evicted for the oldest request, a request that can
    never fit finishes at once with IBR_ENOMEM;
  - residency: a request with a resident geometry skips the set-up and gives
    the same result;
  - the device-memory estimate bounds what a grid really allocates;
  - the schedule autotuner picks one schedule per shape and its solves still
    meet the tolerance (1e-7 of the oracle at residual 1e-8).
"""
import numpy as np
import pytest

from oracle import fft_stokes, ib
from oracle.system import drag
from synthetic import Request, disk_markers, random_quaternion, sphere_markers, ellipsoid_markers

from ._util import flat_fields, gpu_grid, oracle_problem, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import abi as a

    assert torch.cuda.is_available()
    return a


def _mix(seed=77):
    """Small periodic problems of several shapes, body counts, precisions."""
    rng = np.random.default_rng(seed)
    out = []
    for n, nb in ((32, 2), (64, 3), (32, 1), (64, 1)):
        h = 1.0 / n
        cs = [np.array([(i + 0.5) / nb, 0.5]) + rng.uniform(-0.05, 0.05, 2) for i in range(nb)]
        rels = [disk_markers(rng.uniform(3.0, 4.0) * h if nb > 1 else 0.1, h) for _ in range(nb)]
        out.append(Request((n, n), cs, [np.array([1.0, 0, 0, 0])] * nb, rels, rng.standard_normal((nb, 3))))
    for n, nb in ((16, 1), (24, 2)):
        h = 1.0 / n
        cs = [np.array([(i + 0.5) / nb, 0.5, 0.5]) + rng.uniform(-0.05, 0.05, 3) for i in range(nb)]
        rels = [sphere_markers(2.2 * h, 30) if i == 0 else ellipsoid_markers(1.6 * h, 1.5, h) for i in range(nb)]
        out.append(Request((n, n, n), cs, [random_quaternion(rng) for _ in range(nb)], rels,
                           rng.standard_normal((nb, 6))))
    return out


def _opts(abi, tol=1e-10):
    o = abi.solve_opts_default()
    o.tol = tol
    o.max_iters = 400
    return o


def _submit(abi, S, r, prec, opts=None, want_fields=True):
    return S.submit(r.n, r.L, r.centers, r.rels, r.UO, precision=prec, quats=r.quats, opts=opts,
                    want_fields=want_fields)


def _alone(abi, r, prec, tol=1e-10):
    """the same request solved by ibr_solve_coupled on its own grid"""
    wl = r.workload(ib.quat_rotate)
    G = abi.create_grid(r.d, r.n, r.L, precision=prec)
    try:
        for c, q, rel in zip(r.centers, r.quats, r.rels):
            bid = abi.add_body(G, c, quat=q)
            abi.set_markers(G, bid, rel)
        info = abi.solve_coupled(G, r.UO, opts=_opts(abi, tol))
        lam, ft = abi.get_forces(G, r.d)
        ncell = int(np.prod(r.n))
        v, p = np.zeros(r.d * ncell), np.zeros(ncell)
        abi.get_fields(G, v, p)
    finally:
        abi.destroy_grid(G)
    return info, v, p, lam, ft, wl


_ORACLE = {}


def _oracle(key, wl):
    if key not in _ORACLE:
        pr = oracle_problem(wl)
        v, p, lam = fft_stokes.solve_coupled(pr, wl.UO())
        _ORACLE[key] = (flat_fields(v), p.ravel(), lam, drag(pr, lam))
    return _ORACLE[key]


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
def test_mix_equals_alone_and_oracle(abi, prec):
    P = getattr(abi, prec)
    reqs = _mix()
    alone = [_alone(abi, r, P) for r in reqs]
    with abi.Server(slots=4, budget_bytes=32 << 30) as S:
        tickets = [_submit(abi, S, r, P, opts=_opts(abi)) for r in reqs]
        mix = [S.poll(t) for t in tickets]
        st = S.stats()
    assert st["completed"] == len(reqs) and st["running"] == 0 and st["queued"] == 0
    for i, (r, a, m) in enumerate(zip(reqs, alone, mix)):
        info, v, p, lam, ft, wl = a
        # 1e-10 is at the mixed path's attainable true residual for some of these
        # requests: a stop by the stall rule (IBR_ENOTCONV, results readable)
        # within 2x of the tolerance counts as converged; the checks against the
        # oracle below are unchanged
        assert m["status"] == abi.OK or (m["status"] == abi.ENOTCONV and m["rel_res_true"] <= 2e-10), m
        assert m["status"] == info.status
        assert m["iters"] == info.iters
        # the same kernels on the same data in the same order
        assert np.array_equal(m["lam"], lam) and np.array_equal(m["v"], v) and np.array_equal(m["p"], p)
        for x, y in ((m["lam"], lam), (m["ft"], ft), (m["v"], v), (m["p"], p)):
            assert rel_err(x, y) <= 1e-9
        vo, po, lo, fo = _oracle(i, wl)
        assert rel_err(m["v"], vo) < 1e-9 and rel_err(m["p"], po) < 1e-9
        assert rel_err(m["lam"], lo) < 1e-9 and rel_err(m["ft"], fo) < 1e-9
    # several requests ran at the same time
    iv = sorted((m["t_start_ms"], m["t_end_ms"]) for m in mix)
    assert any(iv[k + 1][0] < iv[k][1] for k in range(len(iv) - 1))
    assert len({m["slot"] for m in mix}) > 1


def test_budget_admission_and_eviction(abi):
    reqs = _mix()[:4]
    ests = [abi.estimate_device_bytes(r.d, r.n, [x.shape[0] for x in r.rels], restart=50, n_s=2) for r in reqs]
    budget = int(max(ests) * 1.05)  # one request at a time
    with abi.Server(slots=4, budget_bytes=budget) as S:
        tickets = [_submit(abi, S, r, abi.MIXED, opts=_opts(abi, 1e-8), want_fields=False) for r in reqs]
        res = [S.poll(t) for t in tickets]
        st = S.stats()
    assert all(m["status"] == abi.OK for m in res)
    assert st["peak_reserved_bytes"] <= budget
    assert st["evictions"] >= 1
    iv = sorted((m["t_start_ms"], m["t_end_ms"]) for m in res)
    assert all(iv[k + 1][0] >= iv[k][1] for k in range(len(iv) - 1))  # never two at once


def test_request_that_never_fits_is_rejected(abi):
    r = _mix()[0]
    with abi.Server(slots=2, budget_bytes=1 << 20) as S:
        t = _submit(abi, S, r, abi.MIXED)
        m = S.poll(t, timeout_ms=0.0)
        st = S.stats()
    assert m is not None and m["status"] == abi.ENOMEM and "budget" in m["error"]
    assert st["rejected"] == 1


def test_resident_geometry_skips_setup(abi):
    r = _mix()[1]
    with abi.Server(slots=1, budget_bytes=8 << 30) as S:
        a = S.poll(_submit(abi, S, r, abi.MIXED, opts=_opts(abi)))
        b = S.poll(_submit(abi, S, r, abi.MIXED, opts=_opts(abi)))
        r2 = Request(r.n, r.centers, r.quats, r.rels, -2.0 * r.UO)
        c = S.poll(_submit(abi, S, r2, abi.MIXED, opts=_opts(abi)))
        st = S.stats()
    assert a["reused_grid"] == 0 and b["reused_geometry"] == 1 and c["reused_geometry"] == 1
    assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["v"], b["v"])
    # a new right-hand side on the resident factorised mobility: linear in U
    assert rel_err(c["lam"], -2.0 * a["lam"]) < 1e-9
    assert st["geometry_reused"] == 2 and st["grids_created"] == 1


def test_poll_pending_and_unknown_ticket(abi):
    r = _mix()[3]
    with abi.Server(slots=1, budget_bytes=8 << 30) as S:
        ts = [_submit(abi, S, r, abi.MIXED, opts=_opts(abi), want_fields=False) for _ in range(3)]
        last = S.poll(ts[-1], timeout_ms=0.0)  # None while queued or running
        out = [S.poll(t) for t in ts[:-1]] + [last if last is not None else S.poll(ts[-1])]
        assert all(m["status"] == abi.OK for m in out)
        with pytest.raises(KeyError):
            S.poll(ts[0])
        assert S.h
        rc = abi._lib.ibr_server_poll(S.h, ts[0], 0.0, None, None, None, None, None)
        assert rc == abi.EINVAL


def test_estimate_bounds_device_memory(abi):
    n = (64, 64, 64)
    rel = sphere_markers(0.2, 400)
    est = abi.estimate_device_bytes(3, n, [400], restart=50, n_s=2, precision=abi.MIXED)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    G = abi.create_grid(3, n, (1.0, 1.0, 1.0), precision=abi.MIXED)
    try:
        bid = abi.add_body(G, (0.5, 0.5, 0.5))
        abi.set_markers(G, bid, rel)
        o = _opts(abi, 1e-8)
        abi.solve_coupled(G, np.ones(6), opts=o)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        abi.destroy_grid(G)
    used = free0 - free1
    assert used <= est, (used, est)
    assert used >= 0.6 * est, (used, est)


def test_autotuned_schedule(abi):
    rng = np.random.default_rng(5)
    n = 64
    reqs = []
    for k in range(4):
        cs = [np.array([0.5, 0.5]) + rng.uniform(-0.1, 0.1, 2)]
        reqs.append(Request((n, n), cs, [np.array([1.0, 0, 0, 0])], [disk_markers(0.1, 1.0 / n)],
                            rng.standard_normal((1, 3))))
    with abi.Server(slots=2, budget_bytes=8 << 30, autotune=True) as S:
        ts = [_submit(abi, S, r, abi.MIXED, want_fields=True) for r in reqs]
        out = [S.poll(t) for t in ts]
        st = S.stats()
    assert st["tuned_shapes"] == 1
    assert sum(m["tuned"] for m in out) == 1
    assert len({(m["n_s"], m["mg_pre"], m["mg_post"]) for m in out}) == 1
    for k, (r, m) in enumerate(zip(reqs, out)):
        assert m["status"] == abi.OK and m["rel_res_true"] <= 1e-8 * (1 + 1e-9)
        vo, po, lo, fo = _oracle(("tune", k), r.workload(ib.quat_rotate))
        assert rel_err(m["v"], vo) < 1e-7 and rel_err(m["lam"], lo) < 1e-7 and rel_err(m["ft"], fo) < 1e-7


def test_many_requests_complete(abi):
    reqs = _mix(seed=3) * 4
    with abi.Server(slots=6, budget_bytes=16 << 30) as S:
        ts = [_submit(abi, S, r, abi.MIXED, opts=_opts(abi, 1e-8), want_fields=False) for r in reqs]
        out = [S.poll(t) for t in ts]
        st = S.stats()
    assert all(m["status"] == abi.OK for m in out)
    assert st["completed"] == st["submitted"] == len(reqs)
    assert st["grids_created"] + st["grids_reused"] == len(reqs)
    assert st["grids_created"] <= 4 * 6  # four shapes, at most six of a shape at once
    # identical requests give identical results, whichever slot ran them
    k = len(reqs) // 4
    for i in range(k):
        for j in (i + k, i + 2 * k, i + 3 * k):
            assert np.array_equal(out[i]["lam"], out[j]["lam"])


def test_malformed_requests_are_rejected_at_submit(abi):
    r = _mix()[0]
    with abi.Server(slots=1, budget_bytes=1 << 30) as S:
        with pytest.raises(abi.IbrError) as e:
            S.submit((31, 32), (1.0, 1.0), r.centers, r.rels, r.UO)  # odd cell count
        assert e.value.code == abi.EINVAL
        with pytest.raises(abi.IbrError) as e:
            S.submit(r.n, r.L, r.centers, r.rels, r.UO, eta=0.0)
        assert e.value.code == abi.EINVAL
        assert S.stats()["submitted"] == 0


def test_free_body_and_precisions_through_the_engine(abi):
    # a free body (given force and torque) and FP64 / mixed requests of the same
    # shape in one engine: each result equals the direct solve of that request
    rng = np.random.default_rng(17)
    n = 32
    h = 1.0 / n
    cs = [np.array([0.3, 0.5]), np.array([0.7, 0.52])]
    rels = [disk_markers(3.5 * h, h), disk_markers(3.0 * h, h)]
    UO = rng.standard_normal((2, 3))
    req = Request((n, n), cs, [np.array([1.0, 0, 0, 0])] * 2, rels, UO)
    kin = [abi.PRESCRIBED, abi.FREE]
    direct = {}
    for prec in (abi.MIXED, abi.FP64):
        G = abi.create_grid(2, (n, n), (1.0, 1.0), precision=prec)
        try:
            for c, rel, k in zip(cs, rels, kin):
                b = abi.add_body(G, c, kinematics=k)
                abi.set_markers(G, b, rel)
            abi.solve_coupled(G, UO, opts=_opts(abi))
            direct[prec] = abi.get_forces(G, 2)
        finally:
            abi.destroy_grid(G)
    with abi.Server(slots=2, budget_bytes=4 << 30) as S:
        ts = {prec: S.submit(req.n, req.L, cs, rels, UO, precision=prec, kinematics=kin, opts=_opts(abi))
              for prec in (abi.MIXED, abi.FP64)}
        out = {prec: S.poll(t) for prec, t in ts.items()}
    for prec in (abi.MIXED, abi.FP64):
        assert out[prec]["status"] == abi.OK
        assert np.array_equal(out[prec]["lam"], direct[prec][0])
        assert np.array_equal(out[prec]["ft"], direct[prec][1])
    # the free body's load is balanced: K^T Lambda equals the applied force/torque
    assert np.allclose(out[abi.FP64]["ft"][1], UO[1], rtol=1e-8, atol=1e-10)
