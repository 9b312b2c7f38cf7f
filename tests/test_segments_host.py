"""The segment arithmetic of the CUDA path (ftk_kernels.cuh: segment_of,
segment_of_coords, segment_count), compiled for the host: segments must be
runs of consecutive vertex ids in order -- (t, z, y-block) for whole rows,
(t, z, y, x-window) for rows cut into windows -- since the compaction
writes each segment's faces as one run in face-id order.  Checked on every
vertex of small grids, through the FastDiv and the 64-bit paths."""
import ctypes
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(ROOT, "tests", "sos_host_shim.cu")
    so = os.path.join(str(tmp_path_factory.mktemp("seg")), "seg_shim.so")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", src, "-o", so])
    lib = ctypes.CDLL(so)
    lib.shim_segment.argtypes = [ctypes.c_int] * 8 + [ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    lib.shim_segment.restype = None
    return lib


def _segs(shim, dims, ry, nxb, wx, small):
    nx, ny, nz, nt = dims
    out = (ctypes.c_longlong * 3)()
    res = []
    for g in range(nx * ny * nz * nt):
        shim.shim_segment(nx, ny, nz, nt, ry, nxb, wx, small, g, out)
        res.append((out[0], out[1], out[2]))
    return res


CASES = [
    # (nx, ny, nz, nt), ry, x windows (nxb, wx): whole rows have nxb = 1
    ((7, 5, 1, 3), 2, 1, 7),
    ((9, 6, 4, 2), 4, 1, 9),
    ((10, 4, 1, 3), 1, 4, 3),     # windows of 3 columns, the last one ragged
    ((11, 3, 2, 2), 1, 2, 8),
    ((16, 2, 3, 2), 1, 2, 8),     # windows dividing the row
    ((5, 3, 2, 1), 1, 0, 5),      # nxb = 0 (a blocking made without windows) means whole rows
]


@pytest.mark.parametrize("dims,ry,nxb,wx", CASES)
@pytest.mark.parametrize("small", [1, 0])
def test_segments_are_ordered_runs(shim, dims, ry, nxb, wx, small):
    nx, ny, nz, nt = dims
    res = _segs(shim, dims, ry, nxb, wx, small)
    count = res[0][2]
    windows = max(nxb, 1)
    assert count == nt * nz * -(-ny // ry) * windows
    seg = [a for a, _, _ in res]
    assert all(a == b for a, b, _ in res), "segment_of and segment_of_coords differ"
    assert seg == sorted(seg), "segments out of face-id order"
    assert set(seg) <= set(range(count))
    # each segment is one run of ids covering exactly its rows and columns
    for s, grp in itertools.groupby(enumerate(seg), key=lambda p: p[1]):
        ids = [g for g, _ in grp]
        assert ids == list(range(ids[0], ids[-1] + 1))
    runs = [len(list(grp)) for _, grp in itertools.groupby(seg)]
    assert len(runs) == len(set(seg)), "a segment split into two runs"
    if windows > 1:
        # a windowed segment is one row's window: at most wx columns
        assert max(runs) <= wx and ry == 1
