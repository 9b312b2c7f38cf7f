"""The FP32 Morse-index filters of the CUDA path (the device's accumulation
of S = sum_k w_k (H_k + H_k^T) and its certified sign tests, compiled for the
host) against exact integer arithmetic: whenever a filter certifies an index
it must be the exact one (Sec. 4.1 / Sec. 7 classification, read as the
sign changes of (1, tr S, m2 S, det S)).  Random, wide-range and
near-singular S, and exactly singular S (never certified)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

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
    lib.shim_morse_filter.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.shim_morse_filter.restype = ctypes.c_int
    return lib


def _sgn(v):
    return (v > 0) - (v < 0)


def exact_index(n, w, hs):
    """Exact Morse index from Python integers (-1: det S = 0)."""
    S = [[sum(w[k] * hs[k][a][b] for k in range(n + 1)) for b in range(n)] for a in range(n)]
    if n == 2:
        det = S[0][0] * S[1][1] - S[0][1] * S[1][0]
        if det == 0:
            return -1
        return 1 if det < 0 else (2 if S[0][0] + S[1][1] < 0 else 0)
    tr = S[0][0] + S[1][1] + S[2][2]
    m2 = (S[0][0] * S[1][1] - S[0][1] * S[1][0] + S[0][0] * S[2][2] - S[0][2] * S[2][0]
          + S[1][1] * S[2][2] - S[1][2] * S[2][1])
    det = (S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) - S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0])
           + S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]))
    if det == 0:
        return -1
    prev, changes = 1, 0
    for s in (_sgn(tr), _sgn(m2), _sgn(det)):
        if s != 0:
            changes += s != prev
            prev = s
    return changes


def run_filter(shim, n, w, hs):
    hi = (ctypes.c_longlong * (n + 1))()
    lo = (ctypes.c_ulonglong * (n + 1))()
    for k, v in enumerate(w):
        u = v & ((1 << 128) - 1)
        h = u >> 64
        hi[k] = h - (1 << 64) if h >= 1 << 63 else h
        lo[k] = u & ((1 << 64) - 1)
    flat = [hs[k][a][b] for k in range(n + 1) for a in range(n) for b in range(n)]
    arr = (ctypes.c_longlong * len(flat))(*flat)
    m = ctypes.c_int(0)
    ok = shim.shim_morse_filter(n, hi, lo, arr, ctypes.byref(m))
    return bool(ok), m.value


def _sym(rng, n, mag):
    a = [[0] * n for _ in range(n)]
    for i in range(n):
        for j in range(i, n):
            v = int(rng.integers(-mag, mag + 1))
            a[i][j] = a[j][i] = v
    return a


def _check(shim, n, cases):
    certified = wrong = 0
    for w, hs in cases:
        ok, m = run_filter(shim, n, w, hs)
        if ok:
            certified += 1
            wrong += m != exact_index(n, w, hs)
    return certified, wrong


@pytest.mark.parametrize("n", [2, 3])
def test_random_wide_range(shim, n):
    rng = np.random.default_rng(11 + n)
    wmax_bits = 61 if n == 2 else 93
    cases = []
    for _ in range(4000):
        w = []
        for _ in range(n + 1):
            bits = int(rng.integers(1, wmax_bits + 1))
            mag = int.from_bytes(rng.bytes(16), "little") >> (128 - bits)
            w.append(-mag if rng.integers(0, 2) else mag)
        hs = [_sym(rng, n, 1 << int(rng.integers(0, 34))) for _ in range(n + 1)]
        cases.append((w, hs))
    certified, wrong = _check(shim, n, cases)
    assert wrong == 0
    assert certified > 0.9 * len(cases)


@pytest.mark.parametrize("n", [2, 3])
def test_near_singular(shim, n):
    """S close to a singular matrix: every H_k a multiple of one rank-deficient
    matrix plus a tiny perturbation; most must fall through to the exact path,
    and nothing certified may be wrong."""
    rng = np.random.default_rng(23 + n)
    cases = []
    for _ in range(3000):
        v = [int(rng.integers(-1000, 1001)) for _ in range(n)]
        base = [[v[a] * v[b] for b in range(n)] for a in range(n)]   # rank 1
        w = [int(rng.integers(-(1 << 40), 1 << 40)) for _ in range(n + 1)]
        hs = []
        for k in range(n + 1):
            c = int(rng.integers(-1000, 1001))
            e = _sym(rng, n, int(rng.integers(0, 3)))
            hs.append([[c * base[a][b] + e[a][b] for b in range(n)] for a in range(n)])
        cases.append((w, hs))
    _, wrong = _check(shim, n, cases)
    assert wrong == 0


@pytest.mark.parametrize("n", [2, 3])
def test_exactly_singular_never_certified(shim, n):
    rng = np.random.default_rng(31 + n)
    for _ in range(500):
        v = [int(rng.integers(-1 << 15, 1 << 15)) for _ in range(n)]
        w = [int(rng.integers(-(1 << 50), 1 << 50)) for _ in range(n + 1)]
        hs = []
        for k in range(n + 1):
            c = int(rng.integers(-1000, 1001))
            hs.append([[c * v[a] * v[b] for b in range(n)] for a in range(n)])
        assert exact_index(n, w, hs) == -1
        ok, _ = run_filter(shim, n, w, hs)
        assert not ok
