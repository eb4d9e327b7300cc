"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
declared in include/ibrigid.h, and its argument validation answers without a
GPU.  No compute entry point runs here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ibrigid.h")


@pytest.fixture(scope="module")
def abi():
    from paper_1505_07865_gb300 import build

    build.build()
    from paper_1505_07865_gb300 import abi as a

    return a


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(ibr_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_abi():
    names = _declared()
    for must in ["ibr_create_grid", "ibr_add_body", "ibr_set_markers", "ibr_solve_coupled", "ibr_get_forces",
                 "ibr_get_fields", "ibr_destroy_grid", "ibr_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(abi):
    lib = ctypes.CDLL(abi.LIBPATH)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", abi.LIBPATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ibr_\w+)", out))
    assert set(_declared()) <= exported
    assert set(abi.exported_names()) == set(_declared())


def test_struct_layouts(abi):
    # C layout: double, 7 ints (+4 pad), double, double[9], double
    assert ctypes.sizeof(abi.SolveOpts) == 8 + 7 * 4 + 4 + 8 + 72 + 8
    assert abi.SolveOpts.mob_a_over_h.offset == 40
    assert ctypes.sizeof(abi.SolveInfo) == 4 * 4 + 4 * 8


def test_default_options(abi):
    o = abi.solve_opts_default()
    assert o.tol == 1e-8 and o.restart == 50 and o.n_s == 0 and o.variant == abi.PC_LOWER
    assert o.mg_pre == 2 and o.mg_post == 2 and o.mob_model == abi.MOB_AUTO
    # zero radius and coefficients: the grid kernel's defaults
    assert o.mob_a_over_h == 0.0 and not any(o.mob_coef)


def test_mobility_defaults_are_the_committed_fit(abi):
    # 3-D radii are the paper's (Sec. IV.A); the 2-D App. B sets are the
    # output of the package's fit script (fit_mobility_2d.py, 256^2 fits)
    import json
    import os

    fit = json.load(open(os.path.join(os.path.dirname(abi.__file__), "mobility_fit_2d.json")))
    for kernel, a3 in ((abi.KERNEL_PESKIN4, 1.25), (abi.KERNEL_BKP6, 1.47)):
        aoh, coef = abi.mobility_defaults(3, kernel)
        assert aoh == a3 and not coef.any()
        f = [x for x in fit["fits"] if x["kernel"] == kernel and x["n"] == 256][0]
        aoh, coef = abi.mobility_defaults(2, kernel)
        assert aoh == f["a_over_h"]
        assert list(coef) == f["a"] + f["b"]
    with pytest.raises(abi.IbrError):
        abi.mobility_defaults(2, 5)


@pytest.mark.parametrize("args,msg", [
    ((4, [8, 8], [1, 1]), "dim must be 2 or 3"),
    ((2, [7, 8], [1, 1]), "even"),
    ((2, [8, 8], [1, 2]), "cubes"),
    ((2, [8, 8], [1, 1], [0, 1, 1, 1]), "periodic at both ends"),   # one periodic side, one wall
    ((2, [8, 8], [1, 1], [7, 7, 0, 0]), "bounded by walls"),        # unknown condition
])
def test_create_grid_validation_without_gpu(abi, args, msg):
    with pytest.raises(abi.IbrError) as e:
        abi.create_grid(*args)
    assert e.value.code == abi.EINVAL
    assert msg in abi.last_error()


def test_null_handles_rejected(abi):
    assert abi._lib.ibr_solve_opts_default(None) == abi.EINVAL
    assert abi._lib.ibr_destroy_grid(None) == abi.OK
    assert abi._lib.ibr_set_markers(None, 0, None, 1) == abi.EINVAL
    assert abi._lib.ibr_apply_system(None, None, None) == abi.EINVAL


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "ibrigid.h"
#define F(T, m) printf(#T " " #m " %zu\n", offsetof(T, m))
int main(void) {
    printf("ibr_request size %zu\n", sizeof(ibr_request));
    printf("ibr_result size %zu\n", sizeof(ibr_result));
    printf("ibr_server_stats size %zu\n", sizeof(ibr_server_stats));
    F(ibr_request, eta); F(ibr_request, x_c); F(ibr_request, opts); F(ibr_request, want_fields);
    F(ibr_result, rel_res_true); F(ibr_result, reserved_bytes); F(ibr_result, slot); F(ibr_result, n_bodies);
    F(ibr_server_stats, tuned_shapes);
    return 0;
}
"""


def test_server_struct_layouts_match_c(abi, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        t, m, v = line.split()
        got[(t, m)] = int(v)
    assert got[("ibr_request", "size")] == ctypes.sizeof(abi.Request)
    assert got[("ibr_result", "size")] == ctypes.sizeof(abi.Result)
    assert got[("ibr_server_stats", "size")] == ctypes.sizeof(abi.ServerStats)
    for (t, m), v in got.items():
        if m == "size":
            continue
        cls = {"ibr_request": abi.Request, "ibr_result": abi.Result, "ibr_server_stats": abi.ServerStats}[t]
        assert getattr(cls, m).offset == v, (t, m)


def test_device_memory_estimate_is_consistent(abi):
    # host-only arithmetic: grows with the grid, the markers, the restart and
    # the precision; the Krylov basis dominates large grids
    e = abi.estimate_device_bytes
    base = e(3, (64, 64, 64), [400])
    assert e(3, (128, 128, 128), [400]) > 7 * base
    assert e(3, (64, 64, 64), [800]) > base
    assert e(3, (64, 64, 64), [400], precision=abi.FP64) > base
    # ten more restart vectors: 2 x 10 FP64 system vectors (basis and Z)
    len_ = 4 * 64 ** 3 + 3 * 400
    d10 = e(3, (64, 64, 64), [400], restart=60) - base
    assert abs(d10 - 2 * 10 * 8 * len_) < 0.05 * d10
    # dense mobility blocks: (3 N)^2 entries in FP64 (built) + FP32 (inverse, work)
    dm = e(2, (64, 64), [2000]) - e(2, (64, 64), [1000])
    assert dm > 0
    # the analytic forms give one block per body: one block of 2N costs more
    # than two of N; coupled (one block of all markers while d N <= 6144)
    # two bodies of N cost what one body of 2N does, beyond the limit a block each
    assert e(2, (64, 64), [2000]) - e(2, (64, 64), [1000, 1000]) > 0
    cpl = abi.MOB_AUTO | abi.MOB_COUPLED
    assert e(2, (64, 64), [2000], mob_model=cpl) == e(2, (64, 64), [1000, 1000], mob_model=cpl)
    assert e(2, (64, 64), [4000], mob_model=cpl) - e(2, (64, 64), [2000, 2000], mob_model=cpl) > 0
    with pytest.raises(abi.IbrError):
        e(4, (8, 8), [1])


def test_server_create_without_gpu_fails_cleanly(abi):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(abi.IbrError) as ex:
        abi.Server(slots=2, budget_bytes=1 << 30)
    assert ex.value.code == abi.ECUDA
    assert abi._lib.ibr_server_create(None, 1, 1, 0) == abi.EINVAL
    assert abi._lib.ibr_server_destroy(None) == abi.OK
