"""CPU oracle for isovolume tracking on the simplicial spacetime mesh.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the CPU-baseline leg of
``bench.py``; never by the product path.  It shares no code with the CUDA
path (the field samplers of ``paper_2011_08697_gb300.synth`` hold none of
the method's arithmetic).

Plain statement of the method (paper Sec. 6.1; Algorithm 1, right column):

1. sign        the isovalue test is a 1-D vector field w(u) = f(u) - c whose
               symbolic perturbation is a positive infinitesimal, so vertex
               u is above the level set iff f(u) >= c, below iff f(u) < c
               (no vertex lies on it, no edge in it)
2. edge pass   every 1-simplex (v, v + bits(m)), m a nonempty axis mask, is
               intersected iff its two vertices have different signs
               (C core ``iso_oracle.c``)
3. location    mu = w(v) / (w(v) - w(v + bits(m))) in FP64; the point is
               v + mu bits(m) (linear interpolation along the edge)
4. cell pass   every cell (pentachoron in 3D + time, tetrahedron in 2D +
               time) unites its intersected edges; a piece of the isovolume
               is a component, labelled by its smallest edge id (C core)

Edge ids: g * (2^d - 1) + (m - 1), g = row-major vertex id (x fastest, time
slowest), d = n + 1.  Every function here is pinned by
``tests/test_oracle_iso.py``.
"""
from __future__ import annotations

import numpy as np

from oracle import cp


def _p64(a):
    return cp._p64(a)


def _pd(a):
    import ctypes
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grid_dims(f: np.ndarray):
    """(nx, ny[, nz], nt) of a field laid out f[t][z][y][x] (or f[t][y][x])."""
    return tuple(int(v) for v in f.shape[::-1])


def edge_ids(f: np.ndarray, c: float) -> np.ndarray:
    """Edge pass (Algorithm 1, right column, first loop): ids of the edges
    whose vertices lie on different sides of f = c, in increasing order."""
    f64 = np.ascontiguousarray(np.asarray(f, dtype=np.float32), dtype=np.float64)
    n = f64.ndim - 1
    dims = np.asarray(grid_dims(f64), dtype=np.int64)
    lib = cp.clib()
    cnt = lib.oracle_iso_edges(n, _p64(dims), _pd(f64), float(c), _p64(np.zeros(1, np.int64)), 0)
    ids = np.zeros(max(cnt, 1), dtype=np.int64)
    got = lib.oracle_iso_edges(n, _p64(dims), _pd(f64), float(c), _p64(ids), cnt)
    assert got == cnt
    return ids[:cnt]


def link(f: np.ndarray, c: float, ids: np.ndarray, with_counts: bool = False):
    """Cell pass (Algorithm 1, right column, second loop): label of every
    intersected edge = smallest id of its component.  With ``with_counts``
    also the histogram of intersected edges per cell."""
    f64 = np.ascontiguousarray(np.asarray(f, dtype=np.float32), dtype=np.float64)
    n = f64.ndim - 1
    dims = np.asarray(grid_dims(f64), dtype=np.int64)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    labels = np.zeros(max(len(ids), 1), dtype=np.int64)
    counts = np.zeros(11, dtype=np.int64)
    rc = cp.clib().oracle_iso_link(n, _p64(dims), _pd(f64), float(c), _p64(ids), len(ids), _p64(labels),
                                   _p64(counts))
    if rc != 0:
        raise AssertionError(f"cell pass failed ({rc}): an intersected edge of a cell is not in the edge set")
    labels = labels[:len(ids)]
    return (labels, counts) if with_counts else labels


def locate(f: np.ndarray, c: float, ids: np.ndarray):
    """Base vertex coordinates (x, y, z, t) and in-cell offsets of the
    intersection points: v + mu bits(m), mu = w(v) / (w(v) - w(v + m)),
    w = f - c, in FP64."""
    f64 = np.asarray(f, dtype=np.float32).astype(np.float64)
    n = f64.ndim - 1
    d = n + 1
    E = (1 << d) - 1
    dims = grid_dims(f64)
    flat = f64.ravel()
    ids = np.asarray(ids, dtype=np.int64)
    g = ids // E
    m = ids % E + 1
    coords = []
    rest = g.copy()
    for a in range(d):
        coords.append(rest % dims[a])
        rest //= dims[a]
    stride = [1]
    for a in range(1, d):
        stride.append(stride[-1] * dims[a - 1])
    step = np.zeros_like(g)
    bits = []
    for a in range(d):
        ba = (m >> a) & 1
        bits.append(ba)
        step += ba * stride[a]
    w0 = flat[g] - c
    w1 = flat[g + step] - c
    mu = w0 / (w0 - w1)
    base = np.zeros((len(ids), 4), dtype=np.int64)
    off = np.zeros((len(ids), 4), dtype=np.float64)
    slots = [0, 1, 2][:n] + [3]
    for a in range(d):
        base[:, slots[a]] = coords[a]
        off[:, slots[a]] = mu * bits[a]
    ordinal = ((m >> n) & 1) == 0
    return base, off, ordinal


def track_iso(f: np.ndarray, c: float, with_links: bool = True):
    """The whole isovolume pipeline: edge ids (sorted), base vertices,
    offsets, ordinal flags (edge inside one time slice) and labels."""
    ids = edge_ids(f, c)
    base, off, ordinal = locate(f, c, ids)
    out = {"edge_id": ids, "base": base, "off": off, "ordinal": ordinal}
    if with_links:
        out["label"] = link(f, c, ids)
    return out
