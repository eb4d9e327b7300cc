"""ctypes binding of libibrigid (include/ibrigid.h): argument marshalling only.

Every function here forwards to the C entry point of the same name (without
the ``ibr_`` prefix).  Device arrays are passed as torch CUDA tensors (their
``data_ptr()``), host arrays as NumPy float64 arrays.  Any non-zero status
raises ``IbrError`` carrying ``ibr_last_error()``; ``IBR_ENOTCONV`` and
``IBR_ETIMEOUT`` are returned in ``SolveInfo.status`` instead (the solution is
still readable) unless ``raise_on_notconv`` is set.

There is no fallback: if the shared library is missing, importing this module
raises ``ImportError`` telling how to build it.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libibrigid.so")

OK, EINVAL, ENOMEM, ENOTCONV, ETIMEOUT, ENUMERIC, ECUDA, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PERIODIC, NOSLIP, VELOCITY = 0, 1, 2
KERNEL_PESKIN4 = 4
KERNEL_BKP6 = 6
FP64, MIXED = 0, 1
PRESCRIBED, FREE = 0, 1
PC_LOWER, PC_FULL = 0, 1
MOB_AUTO, MOB_RPY, MOB_FIT2D, MOB_TRUE, MOB_PAIR = 0, 1, 2, 3, 4
MOB_COUPLED = 16  # OR-ed with MOB_AUTO / MOB_RPY / MOB_FIT2D: one block of all markers


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("restart", ctypes.c_int),
        ("max_iters", ctypes.c_int),
        ("n_s", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("mg_pre", ctypes.c_int),
        ("mg_post", ctypes.c_int),
        ("mob_model", ctypes.c_int),
        ("mob_a_over_h", ctypes.c_double),
        ("mob_coef", ctypes.c_double * 9),
        ("time_cap_ms", ctypes.c_double),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("ps_applications", ctypes.c_int),
        ("rel_res_est", ctypes.c_double),
        ("rel_res_true", ctypes.c_double),
        ("ms_setup", ctypes.c_double),
        ("ms_solve", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("steps", ctypes.c_int),
        ("iters_total", ctypes.c_int),
        ("iters_last", ctypes.c_int),
        ("change", ctypes.c_double),
        ("rel_res_last", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EPENDING = -8
RUNNING, QUEUED = 1, 2
SERVER_AUTOTUNE = 1


class Request(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("L", ctypes.c_double * 3),
        ("eta", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("n_bodies", ctypes.c_int),
        ("x_c", ctypes.POINTER(ctypes.c_double)),
        ("quat", ctypes.POINTER(ctypes.c_double)),
        ("kinematics", ctypes.POINTER(ctypes.c_int)),
        ("n_markers", ctypes.POINTER(ctypes.c_int)),
        ("r_body", ctypes.POINTER(ctypes.c_double)),
        ("body_UO", ctypes.POINTER(ctypes.c_double)),
        ("opts", ctypes.POINTER(SolveOpts)),
        ("want_fields", ctypes.c_int),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("rel_res_true", ctypes.c_double),
        ("ms_setup", ctypes.c_double),
        ("ms_solve", ctypes.c_double),
        ("t_submit_ms", ctypes.c_double),
        ("t_start_ms", ctypes.c_double),
        ("t_end_ms", ctypes.c_double),
        ("reserved_bytes", ctypes.c_longlong),
        ("slot", ctypes.c_int),
        ("reused_grid", ctypes.c_int),
        ("reused_geometry", ctypes.c_int),
        ("tuned", ctypes.c_int),
        ("n_s", ctypes.c_int),
        ("mg_pre", ctypes.c_int),
        ("mg_post", ctypes.c_int),
        ("n_markers", ctypes.c_int),
        ("n_bodies", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in (
        "submitted", "completed", "rejected", "queued", "running", "reserved_bytes", "peak_reserved_bytes",
        "budget_bytes", "grids_created", "grids_reused", "geometry_reused", "evictions", "resident_grids",
        "tuned_shapes")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IbrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


if not os.path.exists(LIBPATH):
    raise ImportError(f"{LIBPATH} is not built: run `python -m paper_1505_07865_gb300.build` "
                      "(or __graft_entry__.build()) first")

_lib = ctypes.CDLL(LIBPATH)
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "ibr_solve_opts_default": (ctypes.c_int, [ctypes.POINTER(SolveOpts)]),
    "ibr_create_grid": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _I, _D, _I, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P]),
    "ibr_add_body": (ctypes.c_int, [_P, _D, _D, ctypes.c_int, _I]),
    "ibr_set_markers": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_int]),
    "ibr_set_boundary_velocity": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "ibr_prepare": (ctypes.c_int, [_P, ctypes.POINTER(SolveOpts)]),
    "ibr_solve_coupled": (ctypes.c_int, [_P, _D, _P, ctypes.c_int, ctypes.POINTER(SolveOpts),
                                         ctypes.POINTER(SolveInfo)]),
    "ibr_advance": (ctypes.c_int, [_P, _D, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.POINTER(SolveOpts), ctypes.POINTER(StepInfo)]),
    "ibr_set_velocity": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "ibr_get_forces": (ctypes.c_int, [_P, _D, _D]),
    "ibr_get_fields": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "ibr_get_body_velocities": (ctypes.c_int, [_P, _D, _D]),
    "ibr_sizes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong), _I, _I]),
    "ibr_apply_system": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_spread": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_interp": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_rigid": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_rigid_T": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_mtilde": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "ibr_op_mtilde_solve": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_stokes_pc": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_advect": (ctypes.c_int, [_P, _P, _P]),
    "ibr_op_gemm_tf32x3": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int,
                                          _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, _P]),
    "ibr_op_vcycle": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P, _P, ctypes.c_int]),
    "ibr_destroy_grid": (ctypes.c_int, [_P]),
    "ibr_last_error": (ctypes.c_char_p, []),
    "ibr_op_vcycle_noalloc": (ctypes.c_int, [ctypes.c_int, _I, _D, ctypes.c_double, ctypes.c_double, _P, _P,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "ibr_estimate_device_bytes": (ctypes.c_int, [ctypes.c_int, _I, ctypes.c_int, _I, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
    "ibr_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_longlong, ctypes.c_int]),
    "ibr_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_longlong)]),
    "ibr_server_poll": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(Result), _D, _D,
                                       _D, _D]),
    "ibr_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "ibr_server_destroy": (ctypes.c_int, [_P]),
    "ibr_tuned_smoother_tile": (ctypes.c_int, [ctypes.c_int, _I, _I, _I]),
    "ibr_tuned_vcycle_schedule": (ctypes.c_int, [ctypes.c_int, _I, _I]),
    "ibr_mobility_defaults": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _D, _D]),
    "ibr_launch_count": (ctypes.c_longlong, []),
    "ibr_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "ibr_profile_reset": (ctypes.c_int, []),
    "ibr_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_longlong), _D, _D, _D]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_names():
    return list(_SIGS)


def last_error():
    return _lib.ibr_last_error().decode()


def _check(rc):
    if rc != OK:
        raise IbrError(rc, last_error())
    return rc


def _dptr(a):
    return a.ctypes.data_as(_D)


def _host(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _dev(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch.float64" or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def solve_opts_default():
    o = SolveOpts()
    _check(_lib.ibr_solve_opts_default(ctypes.byref(o)))
    return o


def create_grid(dim, n, L, bc=None, eta=1.0, rho=0.0, dt=0.0, kernel=KERNEL_PESKIN4, precision=MIXED,
                stream=None):
    k = max(3, len(n), len(L), int(dim))
    n_arr = (ctypes.c_int * k)(*(list(n) + [0] * (k - len(n))))
    L_arr = (ctypes.c_double * k)(*(list(L) + [0.0] * (k - len(L))))
    if bc is None:
        bc = [PERIODIC] * (2 * k)
    bc_arr = (ctypes.c_int * (2 * k))(*(list(bc) + [0] * (2 * k - len(bc))))
    h = _P()
    s = None if stream is None else _P(int(stream))
    _check(_lib.ibr_create_grid(ctypes.byref(h), int(dim), n_arr, L_arr, bc_arr, float(eta), float(rho), float(dt),
                                int(kernel), int(precision), s))
    return h


def add_body(grid, x_c, quat=None, kinematics=PRESCRIBED):
    xc = _host(x_c)
    q = None if quat is None else _dptr(_host(quat, 4))
    bid = ctypes.c_int()
    _check(_lib.ibr_add_body(grid, _dptr(xc), q, int(kinematics), ctypes.byref(bid)))
    return bid.value


def set_markers(grid, body_id, r_body):
    r = _host(r_body)
    N = r.shape[0] if r.ndim == 2 else r.size
    _check(_lib.ibr_set_markers(grid, int(body_id), _dptr(r), int(N)))


def set_boundary_velocity(grid, face, values):
    v = _host(values)
    _check(_lib.ibr_set_boundary_velocity(grid, int(face), _dptr(v)))


def prepare(grid, opts=None):
    _check(_lib.ibr_prepare(grid, None if opts is None else ctypes.byref(opts)))


def solve_coupled(grid, body_UO, g=None, opts=None, raise_on_notconv=False):
    uo = _host(body_UO)
    info = SolveInfo()
    if g is None:
        gp, on_dev = None, 0
    elif hasattr(g, "is_cuda"):
        gp, on_dev = _dev(g), 1
    else:
        garr = _host(g)
        gp, on_dev = garr.ctypes.data_as(_P), 0
    rc = _lib.ibr_solve_coupled(grid, _dptr(uo), gp, on_dev, None if opts is None else ctypes.byref(opts),
                                ctypes.byref(info))
    if rc in (ENOTCONV, ETIMEOUT) and not raise_on_notconv:
        return info
    _check(rc)
    return info


def _field_arg(g):
    if g is None:
        return None, 0, None
    if hasattr(g, "is_cuda"):
        return _dev(g), 1, g
    arr = _host(g)
    return arr.ctypes.data_as(_P), 0, arr


def advance(grid, body_UO, nsteps, steady_tol=0.0, g=None, opts=None, raise_on_notconv=False):
    """Time steps (ibr_advance); g: constant body force (host array or CUDA tensor) or None."""
    uo = _host(body_UO)
    info = StepInfo()
    gp, on_dev, _keep = _field_arg(g)
    rc = _lib.ibr_advance(grid, _dptr(uo), gp, on_dev, int(nsteps), float(steady_tol),
                          None if opts is None else ctypes.byref(opts), ctypes.byref(info))
    if rc in (ENOTCONV, ETIMEOUT) and not raise_on_notconv:
        return info
    _check(rc)
    return info


def set_velocity(grid, v):
    vp, on_dev, _keep = _field_arg(v)
    _check(_lib.ibr_set_velocity(grid, vp, on_dev))


def sizes(grid):
    ln = ctypes.c_longlong()
    nm = ctypes.c_int()
    nb = ctypes.c_int()
    _check(_lib.ibr_sizes(grid, ctypes.byref(ln), ctypes.byref(nm), ctypes.byref(nb)))
    return ln.value, nm.value, nb.value


def get_forces(grid, dim):
    _, N, B = sizes(grid)
    lam = np.zeros(N * dim)
    ft = np.zeros(B * (dim + (1 if dim == 2 else 3)))
    _check(_lib.ibr_get_forces(grid, _dptr(lam), _dptr(ft)))
    return lam.reshape(N, dim), ft.reshape(B, -1)


def get_body_velocities(grid, body_UO):
    """Rigid velocities after a solve: body_UO with free bodies' rows replaced."""
    uo = _host(body_UO)
    out = np.zeros_like(uo)
    _check(_lib.ibr_get_body_velocities(grid, _dptr(uo), _dptr(out)))
    return out


def get_fields(grid, v=None, p=None):
    """Copies v (dim face arrays, concatenated) and p into the given buffers:
    NumPy arrays (host) or torch CUDA tensors (device, both)."""
    if v is not None and hasattr(v, "is_cuda"):
        _check(_lib.ibr_get_fields(grid, _dev(v), None if p is None else _dev(p), 1))
    else:
        vp = None if v is None else v.ctypes.data_as(_P)
        pp = None if p is None else p.ctypes.data_as(_P)
        _check(_lib.ibr_get_fields(grid, vp, pp, 0))
    return v, p


def apply_system(grid, x, y):
    _check(_lib.ibr_apply_system(grid, _dev(x), _dev(y)))


def op_spread(grid, lam, f):
    _check(_lib.ibr_op_spread(grid, _dev(lam), _dev(f)))


def op_interp(grid, v, U):
    _check(_lib.ibr_op_interp(grid, _dev(v), _dev(U)))


def op_rigid(grid, UO, V):
    _check(_lib.ibr_op_rigid(grid, _dev(UO), _dev(V)))


def op_rigid_T(grid, lam, FT):
    _check(_lib.ibr_op_rigid_T(grid, _dev(lam), _dev(FT)))


def op_mtilde(grid, body, out):
    _check(_lib.ibr_op_mtilde(grid, int(body), _dev(out)))


def op_mtilde_solve(grid, rhs, out):
    _check(_lib.ibr_op_mtilde_solve(grid, _dev(rhs), _dev(out)))


def op_advect(grid, v, N):
    _check(_lib.ibr_op_advect(grid, _dev(v), _dev(N)))


def op_gemm_tf32x3(A, B, C, alpha=1.0, beta=0.0, stream=None):
    """C = beta C + alpha A B^T on the tensor cores; A [M, K], B [N, K], C [M, N]
    contiguous float32 CUDA tensors (row strides may exceed the widths)."""
    for t in (A, B, C):
        if not (hasattr(t, "is_cuda") and t.is_cuda) or str(t.dtype) != "torch.float32" or t.stride(1) != 1:
            raise TypeError("expected float32 CUDA tensors with unit column stride")
    M, K = A.shape
    N = B.shape[0]
    s = None if stream is None else _P(int(stream))
    _check(_lib.ibr_op_gemm_tf32x3(M, N, K, _P(A.data_ptr()), A.stride(0), _P(B.data_ptr()), B.stride(0),
                                   _P(C.data_ptr()), C.stride(0), float(alpha), float(beta), s))


def op_stokes_pc(grid, r, z):
    _check(_lib.ibr_op_stokes_pc(grid, _dev(r), _dev(z)))


def op_vcycle(grid, sigma, kappa, f, u, k):
    _check(_lib.ibr_op_vcycle(grid, float(sigma), float(kappa), _dev(f), _dev(u), int(k)))


def op_vcycle_noalloc(dim, n, L, sigma, kappa, f, u, k, pre=2, post=2, stream=None):
    """ibr_op_vcycle_noalloc: k V-cycles with the library's static scratch
    (no device allocation); f, u float64 CUDA tensors."""
    n_arr = (ctypes.c_int * 3)(*(list(n) + [0] * (3 - len(n))))
    L_arr = (ctypes.c_double * 3)(*(list(L) + [0.0] * (3 - len(L))))
    s = None if stream is None else _P(int(stream))
    _check(_lib.ibr_op_vcycle_noalloc(int(dim), n_arr, L_arr, float(sigma), float(kappa), _dev(f), _dev(u),
                                      int(k), int(pre), int(post), s))


def destroy_grid(grid):
    _check(_lib.ibr_destroy_grid(grid))


def launch_count():
    return int(_lib.ibr_launch_count())


def profile_enable(on=True):
    _check(_lib.ibr_profile_enable(1 if on else 0))


def profile_reset():
    _check(_lib.ibr_profile_reset())


def profile_read(with_flops=False):
    """{kernel class: (launches, total_ms, total_algorithmic_bytes[, flops])}
    for every class with at least one timed launch."""
    out = {}
    i = 0
    buf = ctypes.create_string_buffer(64)
    while True:
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        fl = ctypes.c_double()
        if _lib.ibr_profile_read(i, buf, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                 ctypes.byref(fl)) != OK:
            break
        if n.value:
            out[buf.value.decode()] = (n.value, ms.value, by.value) + ((fl.value,) if with_flops else ())
        i += 1
    return out


def estimate_device_bytes(dim, n, n_markers, restart=50, n_s=0, precision=MIXED, mob_model=MOB_AUTO):
    """ibr_estimate_device_bytes: device bytes one periodic grid holds in a solve."""
    n_arr = (ctypes.c_int * 3)(*(list(n) + [0] * (3 - len(n))))
    nm = (ctypes.c_int * max(1, len(n_markers)))(*[int(x) for x in n_markers])
    out = ctypes.c_longlong()
    _check(_lib.ibr_estimate_device_bytes(int(dim), n_arr, len(n_markers), nm, int(restart), int(n_s),
                                          int(precision), int(mob_model), ctypes.byref(out)))
    return out.value


class Server:
    """The serving engine (ibr_server_*): submit() queues one periodic
    constrained solve and returns a ticket, poll() collects its result.

    Bodies are given as a list of (x_c, rel[N_b, dim]) with optional quats;
    body_UO is [B, dim + rot].  Argument marshalling only: the engine, its
    admission control and the solves run in the library."""

    def __init__(self, slots=4, budget_bytes=64 << 30, autotune=False):
        self.h = _P()
        _check(_lib.ibr_server_create(ctypes.byref(self.h), int(slots), int(budget_bytes),
                                      SERVER_AUTOTUNE if autotune else 0))
        self._sizes = {}

    def submit(self, n, L, centers, rels, body_UO, eta=1.0, precision=MIXED, quats=None, kinematics=None,
               opts=None, want_fields=False):
        dim = len(n)
        B = len(centers)
        rot = 1 if dim == 2 else 3
        xc = _host(np.asarray(centers, dtype=np.float64).reshape(B, dim))
        nm = np.array([np.asarray(r).reshape(-1, dim).shape[0] for r in rels], dtype=np.int32)
        rb = _host(np.concatenate([np.asarray(r, dtype=np.float64).reshape(-1, dim) for r in rels]))
        uo = _host(np.asarray(body_UO, dtype=np.float64).reshape(B, dim + rot))
        r = Request()
        r.dim = dim
        for a in range(dim):
            r.n[a] = int(n[a])
            r.L[a] = float(L[a])
        r.eta = float(eta)
        r.precision = int(precision)
        r.n_bodies = B
        r.x_c = _dptr(xc)
        qa = None
        if quats is not None:
            qa = _host(np.asarray(quats, dtype=np.float64).reshape(B, 4))
            r.quat = _dptr(qa)
        ka = None
        if kinematics is not None:
            ka = np.ascontiguousarray(np.asarray(kinematics, dtype=np.int32))
            r.kinematics = ka.ctypes.data_as(_I)
        r.n_markers = nm.ctypes.data_as(_I)
        r.r_body = _dptr(rb)
        r.body_UO = _dptr(uo)
        if opts is not None:
            r.opts = ctypes.pointer(opts)
        r.want_fields = 1 if want_fields else 0
        t = ctypes.c_longlong()
        _check(_lib.ibr_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)))
        ncell = int(np.prod(n))
        self._sizes[t.value] = (dim, int(nm.sum()), B, ncell, bool(want_fields))
        return t.value

    def poll(self, ticket, timeout_ms=-1.0):
        """None while pending; else a dict: result fields, 'lam' [N, dim],
        'ft' [B, dim + rot], and 'v', 'p' when the request wanted fields."""
        dim, N, B, ncell, wf = self._sizes[ticket]
        rot = 1 if dim == 2 else 3
        res = Result()
        lam = np.zeros(N * dim)
        ft = np.zeros(B * (dim + rot))
        v = np.zeros(dim * ncell) if wf else None
        p = np.zeros(ncell) if wf else None
        rc = _lib.ibr_server_poll(self.h, int(ticket), float(timeout_ms), ctypes.byref(res), _dptr(lam), _dptr(ft),
                                  None if v is None else _dptr(v), None if p is None else _dptr(p))
        if rc == EPENDING:
            return None
        del self._sizes[ticket]
        out = res.as_dict()
        out["error"] = last_error() if rc != OK else ""
        out["lam"] = lam.reshape(N, dim)
        out["ft"] = ft.reshape(B, dim + rot)
        if wf:
            out["v"], out["p"] = v, p
        return out

    def stats(self):
        st = ServerStats()
        _check(_lib.ibr_server_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            _check(_lib.ibr_server_destroy(self.h))
            self.h = _P()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tuned_smoother_tiles():
    """[(n0, n1, n2, stacked fields, element bytes, by, kz)] picked by the smoother autotuner."""
    out = []
    i = 0
    v = (ctypes.c_int * 5)()
    by, kz = ctypes.c_int(), ctypes.c_int()
    while _lib.ibr_tuned_smoother_tile(i, v, ctypes.byref(by), ctypes.byref(kz)) == OK:
        out.append(tuple(v) + (by.value, kz.value))
        i += 1
    return out


def tuned_vcycle_schedules():
    """[(n0, n1, n2, levels, stacked fields, element bytes, first cluster level or -2)]
    picked by the V-cycle schedule autotuner."""
    out = []
    i = 0
    v = (ctypes.c_int * 6)()
    cl = ctypes.c_int()
    while _lib.ibr_tuned_vcycle_schedule(i, v, ctypes.byref(cl)) == OK:
        out.append(tuple(v) + (cl.value,))
        i += 1
    return out


def mobility_defaults(dim, kernel=KERNEL_PESKIN4):
    """(a/h, [a0..a4, b0..b3]) of the library's analytic M~ for the kernel."""
    aoh = ctypes.c_double()
    c = np.zeros(9)
    _check(_lib.ibr_mobility_defaults(int(dim), int(kernel), ctypes.byref(aoh), _dptr(c)))
    return aoh.value, c
