"""The CUDA path's determinant sign with Simulation of Simplicity (Sec. 4.1),
compiled for the host, against the oracle's generic expansion over all
permutations and perturbation subsets: every matrix with entries in
{-1, 0, 1} (massively degenerate), random small-integer matrices and random
wide-range matrices."""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
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
    lib = ctypes.CDLL(so)
    lib.shim_sos_det_sign.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
    lib.shim_sos_det_sign.restype = ctypes.c_int
    return lib


def _both(shim, n, m):
    a32 = np.ascontiguousarray(m, dtype=np.int32).ravel()
    a64 = np.ascontiguousarray(m, dtype=np.int64).ravel()
    got = shim.shim_sos_det_sign(n, a32.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    want = cp.clib().oracle_sos_det_sign(n, a64.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return got, want


@pytest.mark.parametrize("n", [2, 3])
def test_all_ternary_matrices(shim, n):
    bad = 0
    for vals in itertools.product((-1, 0, 1), repeat=n * n):
        got, want = _both(shim, n, vals)
        bad += got != want
    assert bad == 0


def test_random_matrices(shim):
    rng = np.random.default_rng(5)
    for _ in range(20000):
        n = int(rng.integers(2, 4))
        # 2^20 and 2^20 + 1: either side of the int64 fast path's entry range
        lim = int(rng.choice([2, 3, 1000, 1 << 20, (1 << 20) + 1, 1 << 29]))
        m = rng.integers(-lim, lim + 1, size=n * n)
        # rank-deficient cases: a repeated or zero column
        if rng.random() < 0.3:
            m = m.reshape(n, n)
            m[rng.integers(n)] = m[rng.integers(n)] if rng.random() < 0.5 else 0
            m = m.ravel()
        got, want = _both(shim, n, m)
        assert got == want, (n, m.tolist())
