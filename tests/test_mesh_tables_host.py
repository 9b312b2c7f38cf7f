"""The CUDA path's compile-time mesh tables, built for the host, against the
oracle's mesh (Sec. 3.3): face chains in the same type order (so face ids
agree), and per cell of a unit cube its sides -- those through the base
vertex (faces of the cube) and the one opposite it (a face of the next cube
along the cell's first step), which the linking step relies on."""
import ctypes
import os
import shutil
import subprocess

import pytest

from oracle import cp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(ROOT, "tests", "sos_host_shim.cu")
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "sos_host_shim.so")
    deps = [src, os.path.join(ROOT, "paper_2011_08697_gb300", "csrc", "ftk_device.cuh")]
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(d) for d in deps):
        subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", src, "-o", so])
    return ctypes.CDLL(so)


@pytest.mark.parametrize("n", [2, 3])
def test_face_chains_match_oracle_order(shim, n):
    want = cp.face_types(n)
    buf = (ctypes.c_int * (len(want) * n))()
    T = shim.shim_face_chains(n, buf)
    got = [tuple(buf[i * n + k] for k in range(n)) for i in range(T)]
    assert got == want


@pytest.mark.parametrize("n", [2, 3])
def test_cell_sides_match_oracle(shim, n):
    d = n + 1
    grid = cp.Grid([4] * n, 4)
    base = tuple([1] * d)
    want = set()
    for cell in cp.cell_types(n):
        sides = grid.cell_sides(base, cell)
        own = 0
        far = None
        for b, ch in sides:
            tt = grid.ftype_index[tuple(ch)]
            if tuple(b) == base:
                own |= 1 << tt
            else:
                # the one side not through the base vertex: based one step
                # along the cell's first axis
                assert tuple(b) == grid.add_bits(base, cell[0])
                far = tt
        assert bin(own).count("1") == d and far is not None
        want.add((own, far, cell[0].bit_length() - 1))
    C = len(cp.cell_types(n))
    own = (ctypes.c_ulonglong * C)()
    far = (ctypes.c_int * C)()
    axis = (ctypes.c_int * C)()
    assert shim.shim_cell_table(n, own, far, axis) == C
    got = {(own[i], far[i], axis[i]) for i in range(C)}
    assert got == want
    # ordered by the axis of the first step, C / (n+1) cells per axis
    assert [axis[i] for i in range(C)] == sorted(axis[i] for i in range(C))
