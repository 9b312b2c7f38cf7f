"""Pins of the isovolume oracle (paper Sec. 6.1; Algorithm 1, right column;
Sec. 6.3 synthetic data) against closed forms, brute force and exact
arithmetic -- nothing here re-types the oracle's own formulas.

* the moving plane f = x - alpha t (Sec. 6.3, 21^3 x 12): every intersection
  point lies on x = alpha t, one connected isovolume, and the per-slice
  count of intersected edges is the number of mesh edges crossing one
  x-interval (counted by hand below);
* the mesh's edges are exactly the vertex pairs of its cells (brute force
  over the cell enumeration of cp.Grid), and their number has a closed form;
* a sample equal to the isovalue counts as above (positive perturbation):
  the edge set equals that of the field shifted up by less than the level
  gap, and differs from the field shifted down;
* a cell with k of its d + 1 vertices above has k (d + 1 - k) intersected
  edges: 0, 4 or 6 for a pentachoron, 0, 3 or 4 for a tetrahedron (Sec. 6.1
  cases I and II);
* labels equal the components of a breadth-first search over cells sharing
  intersected edges, labelled by their smallest id;
* locations equal the exact rational crossing of the edge's linear
  interpolant.
"""
import itertools
from collections import deque
from fractions import Fraction

import numpy as np
import pytest

from oracle import cp, iso
from paper_2011_08697_gb300 import synth


def _plane(n, nt, alpha, dims):
    """f = x - alpha t sampled at integer coordinates (float32)."""
    shape = (nt,) + tuple(reversed(dims))
    t = np.arange(nt, dtype=np.float64).reshape((nt,) + (1,) * len(dims))
    x = np.arange(dims[0], dtype=np.float64).reshape((1,) * len(dims) + (dims[0],))
    return (x - alpha * t + np.zeros(shape)).astype(np.float32)


def _per_slice(res, nt):
    return [int(np.sum(res["ordinal"] & (res["base"][:, 3] == k))) for k in range(nt)]


def test_moving_plane_exact_3d():
    # dyadic alpha: every sample, every crossing and x = alpha t are exact
    alpha, n, nt = 0.875, 21, 12
    f = _plane(3, nt, alpha, (n, n, n))
    r = iso.track_iso(f, 0.0)
    pos = r["base"] + r["off"]
    assert np.max(np.abs(pos[:, 0] - alpha * pos[:, 3])) < 1e-12
    assert len(np.unique(r["label"])) == 1
    # slice k > 0: the plane x = alpha k crosses one x-interval per (y, z);
    # the edges through it step along x and optionally y and/or z:
    # x: 21*21, xy: 20*21, xz: 21*20, xyz: 20*20
    per = 21 * 21 + 20 * 21 + 21 * 20 + 20 * 20
    # slice 0: x = 0 is the grid's first column, all samples >= 0: nothing crosses
    assert _per_slice(r, nt) == [0] + [per] * (nt - 1)


def test_moving_plane_paper_alpha_3d():
    # the paper's alpha = 0.9: samples are rounded to float32, points stay
    # on x = alpha t to the rounding of the samples
    alpha, n, nt = 0.9, 21, 12
    f = _plane(3, nt, alpha, (n, n, n))
    r = iso.track_iso(f, 0.0)
    pos = r["base"] + r["off"]
    assert np.max(np.abs(pos[:, 0] - alpha * pos[:, 3])) < 1e-5
    assert len(np.unique(r["label"])) == 1


def test_moving_line_exact_2d():
    alpha, n, nt = 0.625, 17, 9
    f = _plane(2, nt, alpha, (n, n))
    r = iso.track_iso(f, 0.0)
    pos = r["base"] + r["off"]
    assert np.max(np.abs(pos[:, 0] - alpha * pos[:, 3])) < 1e-12
    assert len(np.unique(r["label"])) == 1
    assert _per_slice(r, nt) == [0] + [17 + 16] * (nt - 1)   # x and xy edges


def _cell_vertex_pairs(grid):
    """Every pair of vertices of every cell, as (lower id, higher id)."""
    pairs = set()
    for g in range(grid.nverts):
        base = grid.coords(g)
        for chain in grid.ctypes_:
            if not grid.in_bounds(grid.add_bits(base, chain[-1])):
                continue
            vs = [grid.gid(v) for v in grid.simplex_vertices(base, chain)]
            for a, b in itertools.combinations(vs, 2):
                pairs.add((min(a, b), max(a, b)))
    return pairs


@pytest.mark.parametrize("shape", [(4, 5, 3), (3, 4, 3, 5)])
def test_edges_are_the_cells_vertex_pairs(shape):
    rng = np.random.default_rng(3)
    f = rng.integers(-2, 3, size=shape).astype(np.float32)
    dims = shape[::-1]
    grid = cp.Grid(dims[:-1], dims[-1])
    d = grid.d
    E = (1 << d) - 1
    pairs = _cell_vertex_pairs(grid)
    # closed form: sum over nonempty masks m of prod_a (N_a - m_a)
    total = sum(int(np.prod([dims[a] - ((m >> a) & 1) for a in range(d)])) for m in range(1, E + 1))
    assert len(pairs) == total
    flat = f.ravel().astype(np.float64)
    want = []
    for a, b in pairs:
        if (flat[a] >= 0.5) != (flat[b] >= 0.5):
            ca, cb = grid.coords(a), grid.coords(b)
            m = sum(1 << q for q in range(d) if cb[q] != ca[q])
            want.append(a * E + m - 1)
    assert np.array_equal(iso.edge_ids(f, 0.5), np.array(sorted(want), dtype=np.int64))


@pytest.mark.parametrize("shape", [(5, 7, 6), (4, 5, 6, 7)])
def test_sample_at_isovalue_counts_as_above(shape):
    f = synth.random_levels(shape, seed=11)            # values in {-1, 0, 1}
    assert np.any(f == 0)
    got = iso.edge_ids(f, 0.0)
    up = iso.edge_ids(f + np.float32(0.25), 0.0)       # no sample at 0, same order
    down = iso.edge_ids(f - np.float32(0.25), 0.0)
    assert np.array_equal(got, up)
    assert not np.array_equal(got, down)


@pytest.mark.parametrize("shape,levels", [((6, 7, 8), (-1.0, 0.0, 1.0)), ((4, 6, 5, 7), (-1.0, 0.0, 1.0)),
                                          ((5, 9, 8, 7), (-2.0, -1.0, 0.0, 1.0, 2.0))])
def test_cells_have_case_one_or_two(shape, levels):
    f = synth.random_levels(shape, levels=levels, seed=2)
    ids = iso.edge_ids(f, 0.0)
    _, counts = iso.link(f, 0.0, ids, with_counts=True)
    d = len(shape)
    allowed = {k * (d + 1 - k) for k in range(d + 2)}   # {0, 4, 6} or {0, 3, 4}
    assert counts.sum() > 0
    assert set(np.nonzero(counts)[0].tolist()) <= allowed
    assert counts[max(allowed)] > 0 and counts[d] > 0


def _bfs_labels(f, c):
    """Components of intersected edges joined through shared cells, by a
    breadth-first search written independently of the oracle."""
    dims = f.shape[::-1]
    grid = cp.Grid(dims[:-1], dims[-1])
    d = grid.d
    E = (1 << d) - 1
    flat = f.ravel().astype(np.float64)
    above = flat >= c
    adj = {}
    for g in range(grid.nverts):
        base = grid.coords(g)
        for chain in grid.ctypes_:
            if not grid.in_bounds(grid.add_bits(base, chain[-1])):
                continue
            vs = [grid.gid(v) for v in grid.simplex_vertices(base, chain)]
            hit = []
            for a, b in itertools.combinations(sorted(vs), 2):
                if above[a] != above[b]:
                    ca, cb = grid.coords(a), grid.coords(b)
                    m = sum(1 << q for q in range(d) if cb[q] != ca[q])
                    hit.append(a * E + m - 1)
            for e in hit:
                adj.setdefault(e, set()).update(hit)
    label = {}
    for s in sorted(adj):
        if s in label:
            continue
        label[s] = s
        todo = deque([s])
        while todo:
            u = todo.popleft()
            for v in adj[u]:
                if v not in label:
                    label[v] = s
                    todo.append(v)
    return label


@pytest.mark.parametrize("shape,seed", [((5, 6, 7), 0), ((4, 5, 4, 6), 1), ((3, 6, 5, 4), 4)])
def test_labels_match_breadth_first_search(shape, seed):
    f = synth.random_levels(shape, seed=seed)
    r = iso.track_iso(f, 0.0)
    want = _bfs_labels(f, 0.0)
    assert sorted(want) == r["edge_id"].tolist()
    assert [want[int(e)] for e in r["edge_id"]] == r["label"].tolist()


def test_locations_are_exact_crossings():
    rng = np.random.default_rng(9)
    f = rng.normal(size=(4, 5, 6, 7)).astype(np.float32)
    c = 0.125
    r = iso.track_iso(f, c, with_links=False)
    flat = f.ravel()
    dims = f.shape[::-1]
    stride = np.cumprod((1,) + dims[:-1])
    for i in rng.choice(len(r["edge_id"]), size=200, replace=False):
        b, o = r["base"][i], r["off"][i]
        g = int(sum(int(b[[0, 1, 2, 3][a]]) * int(stride[a]) for a in range(4)))
        m = int(r["edge_id"][i] % 15) + 1
        h = g + int(sum(int(stride[a]) for a in range(4) if (m >> a) & 1))
        w0 = Fraction(float(flat[g])) - Fraction(c)
        w1 = Fraction(float(flat[h])) - Fraction(c)
        mu = w0 / (w0 - w1)
        assert 0 <= mu <= 1
        # the linear interpolant is exactly c at mu
        assert Fraction(float(flat[g])) + mu * (Fraction(float(flat[h])) - Fraction(float(flat[g]))) == Fraction(c)
        for a in range(4):
            want = float(mu) if (m >> a) & 1 else 0.0
            assert abs(o[a] - want) < 1e-12


def _two_spheres(sep, n=24, nt=6, r=4.0):
    """f = distance to the nearer of two centres moving along x, level r:
    two spherical shells; they touch once the centres are closer than 2 r."""
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    out = np.zeros((nt, n, n, n), dtype=np.float32)
    for t in range(nt):
        a = np.array([n / 2 - sep(t) / 2, n / 2, n / 2])
        b = np.array([n / 2 + sep(t) / 2, n / 2, n / 2])
        da = np.sqrt((x - a[0]) ** 2 + (y - a[1]) ** 2 + (z - a[2]) ** 2)
        db = np.sqrt((x - b[0]) ** 2 + (y - b[1]) ** 2 + (z - b[2]) ** 2)
        out[t] = np.minimum(da, db)
    return out, r


def test_isovolume_pieces_split_and_merge():
    f, r = _two_spheres(lambda t: 14.0)          # always apart: two pieces
    res = iso.track_iso(f, r)
    assert len(np.unique(res["label"])) == 2
    f, r = _two_spheres(lambda t: 14.0 - 2.0 * t)   # the shells meet at t >= 3: one piece
    res = iso.track_iso(f, r)
    assert len(np.unique(res["label"])) == 1
