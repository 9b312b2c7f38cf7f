"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/*.h declares; argument errors come back as
status codes before any device work."""
import ctypes
import glob
import os
import re

import pytest

from paper_2011_08697_gb300 import build, ftk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return ftk.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ftk_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert len(declared) >= 16
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(ftk.EXPORTS) <= declared


def test_version_and_status_strings(L):
    assert "sm_103a" in ftk.ftk_version()
    for s in range(9):
        assert L.ftk_status_string(s)
    p = ftk.make_params()
    assert p.quant_shift == 20 and p.flags == 0 and p.spacing[0] == 1.0


def test_record_layout_matches_header():
    src = open(os.path.join(ROOT, "include", "ftk.h")).read()
    assert "56 bytes" in src
    assert ftk.CP_DTYPE.itemsize == 56
    assert ctypes.sizeof(ftk.ftk_params) == 8 * 3 * 2 + 16 + 8 + 8


@pytest.mark.parametrize("args,status", [
    ((4, 8, 8, 8, 4), 1),       # ndim must be 2 or 3
    ((2, 1, 8, 1, 4), 1),       # extent < 2
    ((3, 8, 8, 1, 4), 1),       # 3D needs nz >= 2
    ((2, 8, 8, 1, 0), 1),       # nt >= 1
])
def test_plan_create_argument_errors(L, args, status):
    h = ctypes.c_void_p()
    p = ftk.make_params()
    got = L.ftk_plan_create(*args, ctypes.byref(p), ctypes.byref(h))
    assert got == status
    assert not h.value
    assert L.ftk_last_error()


def test_bad_params_rejected(L):
    h = ctypes.c_void_p()
    p = ftk.make_params(quant_shift=99)
    assert L.ftk_plan_create(2, 8, 8, 1, 4, ctypes.byref(p), ctypes.byref(h)) == 1
    p = ftk.make_params(flags=0x80)
    assert L.ftk_plan_create(2, 8, 8, 1, 4, ctypes.byref(p), ctypes.byref(h)) == 1


def test_null_pointers_rejected(L):
    out = ctypes.c_void_p()
    assert L.ftk_track_cp2d(None, 8, 8, 4, None, ctypes.byref(out), None) == 1
    assert not out.value
    assert L.ftk_plan_execute(None, None, None) == 1
    assert L.ftk_plan_destroy(None) == 0
    L.ftk_result_free(None)


@pytest.mark.parametrize("dims", [(2, 6000, 8, 1), (2, 20001, 3, 1), (3, 1030, 5, 4), (3, 4099, 3, 3),
                                  (2, 4096, 16, 1), (3, 1024, 8, 8)])
def test_any_row_width_is_accepted(L, dims):
    """Rows wider than the streaming kernels take (2D: 4096 floats, 3D: 1024)
    go to the tiled kernel, cut into x windows where a row exceeds its tile:
    the host-side blocking accepts every width (no device work here)."""
    p = ftk.make_params()
    out = ctypes.c_uint64(0)
    st = L.ftk_stream_footprint(dims[0], dims[1], dims[2], dims[3], ctypes.byref(p), ctypes.byref(out))
    assert st == 0, L.ftk_last_error().decode()
    assert out.value > 0
