"""Pins for the oracle's quantiser, gradient, location, classification,
linking and streaming semantics (paper Sec. 3.2, Sec. 4)."""
import itertools
import math
from collections import defaultdict, deque
from fractions import Fraction

import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth


# ---------------------------------------------------------------- quantise
def test_quantise_round_half_even_and_range():
    s = 2.0 ** -20
    f = np.array([0.5 * s, 1.5 * s, 2.5 * s, -0.5 * s, -1.5 * s, 0.25 * s, 3.0], np.float32)
    assert list(cp.quantise(f, 20)) == [0, 2, 2, 0, -2, 0, 3 << 20]
    with pytest.raises(cp.OracleRangeError):
        cp.quantise(np.array([300.0], np.float32), 20)   # 300 * 2^20 > 2^28
    with pytest.raises(cp.OracleRangeError):
        cp.quantise(np.array([np.nan], np.float32), 20)


def test_gradient_rule_and_linear_exactness():
    F = np.array([[0, 1, 4, 9, 16]], dtype=np.int64)[None]     # (t, y, x)
    G = cp.gradient(np.repeat(F, 2, axis=1), 2)
    assert list(G[0, 0, :, 0]) == [2, 4, 8, 12, 14]             # x: 2(1-0), 4-0, 9-1, 16-4, 2(16-9)
    assert np.all(G[..., 1] == 0)                                # y: constant rows
    # a linear field has the exact constant gradient 2*slope everywhere
    x = np.arange(6)
    y = np.arange(5)
    z = np.arange(4)
    lin = (3 * x[None, None, :] - 5 * y[None, :, None] + 7 * z[:, None, None])[None]
    G3 = cp.gradient(lin.astype(np.int64), 3)
    assert np.all(G3[..., 0] == 6) and np.all(G3[..., 1] == -10) and np.all(G3[..., 2] == 14)
    H = cp.hessian(G3, 3)
    assert np.all(H == 0)


# ------------------------------------------------------------ classification
@pytest.mark.parametrize("S,want", [
    ([[1, 0], [0, 1]], 0), ([[-1, 0], [0, -1]], 2), ([[1, 0], [0, -1]], 1),
    ([[0, 1], [1, 0]], 1), ([[2, 1], [1, 2]], 0), ([[1, 2], [2, 1]], 1),
    ([[1, 1], [1, 1]], -1), ([[0, 0], [0, 0]], -1),
    ([[1, 0, 0], [0, 1, 0], [0, 0, 1]], 0), ([[-1, 0, 0], [0, -1, 0], [0, 0, -1]], 3),
    ([[1, 0, 0], [0, -1, 0], [0, 0, -1]], 2), ([[-1, 0, 0], [0, 1, 0], [0, 0, 1]], 1),
    ([[0, 1, 0], [1, 0, 0], [0, 0, 1]], 1), ([[1, 0, 0], [0, 0, 0], [0, 0, 1]], -1),
])
def test_morse_index_hand_built(S, want):
    assert cp.morse_index(S) == want


def test_morse_index_vs_eigenvalues():
    rng = np.random.default_rng(5)
    for n in (2, 3):
        for _ in range(300):
            A = rng.integers(-50, 51, size=(n, n))
            S = A + A.T
            w = np.linalg.eigvalsh(S.astype(np.float64))
            if np.min(np.abs(w)) < 1e-6:
                continue
            assert cp.morse_index(S.tolist()) == int(np.sum(w < 0))
    # huge entries (as produced by the weighted Hessian) stay exact
    big = 1 << 90
    assert cp.morse_index([[big, 1], [1, -big]]) == 1
    assert cp.morse_index([[big, big - 1], [big - 1, big]]) == 0


def test_classify_weighting():
    """S = sign(D) sum_k D_k (H_k + H_k^T): with all-negative D_k and a
    positive definite Hessian the type is still a minimum."""
    Hs = [[[2, 0], [0, 2]]] * 3
    assert cp.classify([-1, -2, -3], Hs) == 0
    assert cp.classify([1, 2, 3], [[[-2, 0], [0, -2]]] * 3) == 2


# ----------------------------------------------------------------- location
def test_barycentric_solves_eq1():
    rng = np.random.default_rng(9)
    for n in (2, 3):
        for _ in range(100):
            V = rng.integers(-100, 101, size=(n + 1, n)).tolist()
            mu, D = cp.barycentric(V)
            if sum(D) == 0:
                continue
            assert sum(mu) == 1
            for r in range(n):
                assert sum(mu[k] * V[k][r] for k in range(n + 1)) == 0
    mu, _ = cp.barycentric([[0, 0], [0, 0], [0, 0]])
    assert mu == [Fraction(1, 3)] * 3


# ------------------------------------------------- moving minimum (Sec. 4.4)
@pytest.mark.parametrize("ndim,n,nt,x0,d", [
    (2, 21, 8, (10, 10), (0.25, -0.5)),
    (2, 21, 8, (10, 10), (0.5, 0.5)),        # passes through grid vertices
    (2, 21, 6, (10, 10), (0.0, 0.75)),       # moves along a grid line
    (3, 13, 4, (6, 6, 6), (0.25, -0.5, 0.75)),
    (3, 13, 4, (6, 6, 6), (0.5, 0.5, 0.0)),
    (3, 21, 3, (10, 10, 10), (-0.25, 0.5, 0.5)),   # the paper's 21^3 domain
])
def test_moving_minimum_closed_form(ndim, n, nt, x0, d):
    """f = |x - (x0 + d t)|^2: one trajectory, exactly one ordinal puncture per
    slice at x0 + d k, every puncture on the line, every type a minimum."""
    f = synth.moving_minimum(n, nt, x0, d, ndim)
    r = cp.track(f, shift=17)
    assert len(np.unique(r["label"])) == 1
    x0 = np.asarray(x0, float)
    d = np.asarray(d, float)
    pos = r["base"].astype(float) + r["off"]
    for i in range(len(r["face_id"])):
        t = pos[i, 3]
        assert np.allclose(pos[i, :ndim], x0 + d * t, atol=1e-9)
    for k in range(nt):
        sel = (r["ordinal"] == 1) & (r["base"][:, 3] == k)
        assert sel.sum() == 1
        assert np.allclose(pos[sel][0, :ndim], x0 + d * k, atol=1e-12)
    assert np.all(r["morse"] == 0)


# --------------------------------------------- pairing invariant (Sec. 4.3)
@pytest.mark.parametrize("shape,seed", [((4, 6, 5), 0), ((5, 5, 5), 1), ((3, 4, 4, 4), 2),
                                        ((3, 3, 5, 4), 3)])
def test_pairing_invariant_on_degenerate_fields(shape, seed):
    """Under SoS every spacetime cell has 0 or 2 punctured sides, even on
    fields whose gradients are massively degenerate ({-1,0,1} samples)."""
    f = synth.random_levels(shape, seed=seed)
    r = cp.track(f)          # link() raises PairingError on a violation
    assert len(r["face_id"]) > 0


def _all_cells_components(grid, S):
    """Alg. 1 taken literally: visit every cell of the mesh, pair its
    punctured sides, then BFS the pairing graph."""
    adj = defaultdict(set)
    for gid in range(grid.nverts):
        base = grid.coords(gid)
        for cc in grid.ctypes_:
            vs = grid.simplex_vertices(base, cc)
            if not all(grid.in_bounds(v) for v in vs):
                continue
            hit = [grid.face_id(sb, sc) for sb, sc in grid.cell_sides(base, cc)]
            hit = [h for h in hit if h in S]
            assert len(hit) in (0, 2)
            if hit:
                adj[hit[0]].add(hit[1])
                adj[hit[1]].add(hit[0])
    label = {}
    for s in sorted(S):
        if s in label:
            continue
        comp = []
        q = deque([s])
        label[s] = None
        while q:
            u = q.popleft()
            comp.append(u)
            for v in adj[u]:
                if v not in label:
                    label[v] = None
                    q.append(v)
        m = min(comp)
        for u in comp:
            label[u] = m
    return label


@pytest.mark.parametrize("shape,seed", [((4, 6, 5), 4), ((3, 3, 4, 4), 5)])
def test_link_equals_all_cells_bfs(shape, seed):
    f = synth.random_levels(shape, levels=(-1.0, -0.5, 0.0, 0.5, 1.0), seed=seed)
    r = cp.track(f, with_types=False)
    S = set(int(x) for x in r["face_id"])
    want = _all_cells_components(r["grid"], S)
    assert {int(a): int(b) for a, b in zip(r["face_id"], r["label"])} == want


# --------------------------------------------- spiral woven (Sec. 4.4)
def _spiral_critical_points(t, lim=4.0):
    """Closed-form critical points of cos(u) sin(w), (u, w) = R(t)(x, y):
    extrema at u = k pi, w = pi/2 + m pi (f = +-1), saddles at
    u = pi/2 + k pi, w = m pi.  Returns [(x, y, morse index)]."""
    out = []
    c, s = math.cos(t), math.sin(t)
    for k in range(-3, 4):
        for m in range(-3, 4):
            for kind in ("ext", "sad"):
                if kind == "ext":
                    u, w = k * math.pi, math.pi / 2 + m * math.pi
                    val = math.cos(u) * math.sin(w)
                    idx = 2 if val > 0 else 0
                else:
                    u, w = math.pi / 2 + k * math.pi, m * math.pi
                    idx = 1
                x = u * c + w * s
                y = -u * s + w * c
                if abs(x) <= lim and abs(y) <= lim:
                    out.append((x, y, idx))
    return out


def test_spiral_woven_closed_form_per_slice():
    """32^2 x 10 spiral woven (no noise): per ordinal slice, the punctures
    away from the boundary are the closed-form critical points, with the
    closed-form types, to within the O(h^2) discretisation error."""
    n, nt = 32, 10
    f = synth.spiral_woven(n, nt)
    r = cp.track(f)
    h = 8.0 / (n - 1)
    lo, hi = -4.0 + 2 * h, 4.0 - 2 * h
    tol = 0.35 * h
    ts = np.linspace(0.0, 1.0, nt)
    for k in range(nt):
        sel = (r["ordinal"] == 1) & (r["base"][:, 3] == k)
        pos = -4.0 + h * (r["base"][sel][:, :2] + r["off"][sel][:, :2])
        types = r["morse"][sel]
        cps = [c for c in _spiral_critical_points(ts[k]) if lo < c[0] < hi and lo < c[1] < hi]
        inner = [(p, ty) for p, ty in zip(pos, types) if lo < p[0] < hi and lo < p[1] < hi]
        assert len(cps) >= 8
        for (x, y, idx) in cps:
            dist = [np.hypot(p[0] - x, p[1] - y) for p, _ in inner]
            j = int(np.argmin(dist))
            assert dist[j] < tol, (k, x, y, dist[j])
            assert inner[j][1] == idx
        # and nothing spurious inside the band away from the closed-form points
        for p, ty in inner:
            d = min(np.hypot(p[0] - c[0], p[1] - c[1]) for c in _spiral_critical_points(ts[k], 4.5))
            assert d < tol


# ------------------------------------------------ streaming (Sec. 3.2)
def test_stream_deltas_partition_and_final_labels():
    f = synth.spiral_woven(24, 7)
    r = cp.track(f)
    g = r["grid"]
    ids = [int(x) for x in r["face_id"]]
    pushes = defaultdict(list)
    for fid in ids:
        pushes[cp.stream_push_index(g, fid)].append(fid)
    assert sorted(x for v in pushes.values() for x in v) == ids
    assert set(pushes) <= set(range(7))
    final = cp.stream_labels(g, ids, 6)
    assert final == {int(a): int(b) for a, b in zip(r["face_id"], r["label"])}
    # provisional labels only decrease as slices arrive, never below final
    prev = {}
    for k in range(7):
        lab = cp.stream_labels(g, ids, k)
        for fid, l in lab.items():
            assert l <= fid and l >= final[fid]
            if fid in prev:
                assert l <= prev[fid]
        prev = lab
