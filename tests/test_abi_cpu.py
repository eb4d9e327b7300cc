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
