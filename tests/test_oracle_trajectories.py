"""Pins of the oracle's ordered trajectories and time slices (paper Sec. 4.1:
a trajectory is a PL curve through spacetime, sliced at t = t0).

* Moving minimum (Sec. 4.4): f = |x - (x0 + d t)|^2 has the exact gradient
  2 (x - x0 - d t) at every interior vertex (central differences of a
  quadratic are exact), which is linear in space and time, so the PL
  trajectory is exactly the line x0 + d t: one open polyline, and its slice
  at any t inside the time range is the single point x0 + d t.
* Structure on degenerate and smooth fields: every puncture appears once;
  consecutive points share a spacetime cell with two punctured sides (the
  pairs come from the oracle's cell enumeration); a trajectory is closed iff
  it has no end; paths start at their smaller end; slices are points on
  their segments at the requested time.
"""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth


def _trajs(f, shift=20):
    r = cp.track(f, shift=shift)
    return r, cp.trajectories(r["grid"], r["face_id"], r["label"])


@pytest.mark.parametrize("ndim,n,nt,x0,d,shift", [
    (2, 21, 8, (10, 10), (0.5, 0.5), 17),
    (2, 21, 6, (9, 11), (0.75, -0.25), 17),
    (3, 13, 4, (6, 6, 6), (0.25, -0.5, 0.75), 17),
])
def test_moving_minimum_polyline_is_the_line(ndim, n, nt, x0, d, shift):
    f = synth.moving_minimum(n, nt, x0, d, ndim)
    r, trajs = _trajs(f, shift)
    assert len(trajs) == 1
    order, closed = trajs[0]
    assert not closed and sorted(order) == sorted(int(x) for x in r["face_id"])
    pos = cp.positions(r)
    rng = np.random.default_rng(ndim * 100 + nt)
    for t0 in list(rng.uniform(0.0, nt - 1.0, size=12)) + [0.5, 1.0, 2.25]:
        pts = cp.slice_trajectories(trajs, pos, float(t0))
        assert len(pts) == 1, (t0, pts)
        want = [x0[a] + d[a] * t0 for a in range(ndim)] + [0.0] * (3 - ndim)
        assert np.allclose(pts[0][3], want, atol=1e-9), (t0, pts[0][3], want)


@pytest.mark.parametrize("make", [
    lambda: synth.random_levels((5, 13, 22), seed=6),
    lambda: synth.random_levels((4, 5, 6, 7), seed=8),
    lambda: synth.spiral_woven(40, 7, sigma=0.02, seed=2),
    lambda: synth.gaussian_blobs((20, 18, 16), 5, nblobs=8, seed=3, sigma_range=(2.0, 5.0)),
])
def test_polyline_structure(make):
    f = make()
    r, trajs = _trajs(f)
    g = r["grid"]
    ids = [int(x) for x in r["face_id"]]
    pairs = set()
    for a, b in cp.cell_pairs(g, ids):
        pairs.add((min(a, b), max(a, b)))
    seen = []
    for order, closed in trajs:
        seen += order
        for a, b in zip(order, order[1:]):
            assert (min(a, b), max(a, b)) in pairs
        deg = {x: 0 for x in order}
        for a, b in pairs:
            if a in deg:
                deg[a] += 1
                deg[b] += 1
        ends = [x for x in order if deg[x] < 2]
        assert closed == (not ends)
        if closed:
            assert (min(order[0], order[-1]), max(order[0], order[-1])) in pairs
            assert order[0] == min(order)
        else:
            assert order[0] == min(ends) and order[-1] in ends
    assert sorted(seen) == ids
    assert len(trajs) == len(np.unique(r["label"]))
    # slices: each point lies on its segment, at the requested time
    pos = cp.positions(r)
    nt = f.shape[0]
    for t0 in (0.37, nt / 2.0 - 0.21, nt - 1.5):
        for lab, a, b, xyz in cp.slice_trajectories(trajs, pos, t0):
            pa, pb = np.asarray(pos[a]), np.asarray(pos[b])
            lo, hi = min(pa[3], pb[3]), max(pa[3], pb[3])
            assert lo <= t0 <= hi
            s = (t0 - pa[3]) / (pb[3] - pa[3])
            assert np.allclose(xyz, (pa + s * (pb - pa))[:3])


def _fake(types, closed=False, times=None):
    order = list(range(100, 100 + len(types)))
    ts = times if times is not None else list(range(len(types)))
    pos = {f: (0.0, 0.0, 0.0, float(t)) for f, t in zip(order, ts)}
    morse = dict(zip(order, types))
    return [(order, closed)], pos, morse


@pytest.mark.parametrize("types,closed,h,want", [
    ([0, 0, 0, 1, 0, 0, 0], False, 2, [0, 0, 0, 0, 0, 0, 0]),     # a lone flip inside a run
    ([0, 0, 1, 1, 0, 0], False, 2, [0, 0, 1, 1, 0, 0]),           # two flips: windows disagree
    ([1, 0, 0, 0, 0], False, 2, [1, 0, 0, 0, 0]),                 # path ends keep their type
    ([1, 1, 1, 1, 1, 0], True, 2, [1, 1, 1, 1, 1, 1]),            # loops wrap around
    ([2, 0, 2], False, 1, [2, 2, 2]),
    ([2, 0, 2], True, 1, [2, 2, 2]),                              # loop of 3, h = 1: both neighbours agree
    ([2, 0, 2, 0], True, 2, [2, 0, 2, 0]),                        # a loop of 2h points is left alone
    ([-1, 1, -1, 1, 1, 1, 1], False, 2, [-1, 1, -1, 1, 1, 1, 1]),
    ([1, 1, -1, 1, 1], False, 2, [1, 1, 1, 1, 1]),               # a degenerate type is smoothed too
])
def test_type_smoothing_rule(types, closed, h, want):
    trajs, pos, morse = _fake(types, closed)
    (order, cl, got), = cp.filter_trajectories(trajs, pos, morse, half_window=h)
    if closed and len(types) <= 2 * h:
        assert got == types
    else:
        assert got == want


def test_filters_by_duration_points_and_loops():
    f = synth.moving_minimum(21, 8, (10, 10), (0.5, 0.5), 2)
    r, trajs = _trajs(f, 17)
    pos = cp.positions(r)
    morse = dict(zip(r["face_id"].tolist(), r["morse"].tolist()))
    assert len(cp.filter_trajectories(trajs, pos, morse, min_duration=7.0)) == 1     # spans t = 0 .. 7
    assert len(cp.filter_trajectories(trajs, pos, morse, min_duration=7.001)) == 0
    n = len(trajs[0][0])
    assert len(cp.filter_trajectories(trajs, pos, morse, min_points=n)) == 1
    assert len(cp.filter_trajectories(trajs, pos, morse, min_points=n + 1)) == 0
    # loops: a degenerate field has closed trajectories; dropping them keeps the rest
    g = synth.random_levels((5, 13, 22), seed=6)
    r, trajs = _trajs(g)
    pos = cp.positions(r)
    morse = dict(zip(r["face_id"].tolist(), r["morse"].tolist()))
    nloops = sum(1 for _, c in trajs if c)
    assert nloops > 0
    kept = cp.filter_trajectories(trajs, pos, morse, drop_loops=True)
    assert len(kept) == len(trajs) - nloops and not any(c for _, c, _ in kept)
