"""Ordered trajectories and time slices from the CUDA path (through the C
ABI) against the oracle: the same polylines point for point (face ids in
path order, closed flags, trajectory order) and the same slice crossings
(segments, labels) with positions within 1e-5 of a grid spacing."""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

from parity_util import OFF_TOL, compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2011_08697_gb300 import build, ftk
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ftk


CASES = [
    ("spiral_32x32x10", lambda: synth.spiral_woven(32, 10), 20),
    ("levels2d_37x23x5", lambda: synth.random_levels((5, 23, 37), seed=1), 20),
    ("stream_levels_36x23x5", lambda: synth.random_levels((5, 23, 36), seed=13), 20),
    ("levels3d_11x9x7x4", lambda: synth.random_levels((4, 7, 9, 11), seed=4), 20),
    ("s3_levels_8x9x7x4", lambda: synth.random_levels((4, 7, 9, 8), seed=21), 20),
    ("blobs3d_40x36x33x5", lambda: synth.gaussian_blobs((40, 36, 33), 5, nblobs=12, seed=7,
                                                         sigma_range=(2.0, 6.0)), 20),
    ("minimum2d", lambda: synth.moving_minimum(21, 8, (10, 10), (0.5, 0.5), 2), 17),
    ("minimum3d", lambda: synth.moving_minimum(13, 4, (6, 6, 6), (0.25, -0.5, 0.75), 3), 17),
    ("spiral_noisy_256x256x16", lambda: synth.spiral_woven(256, 16, sigma=1e-3, seed=0), 20),
    ("tiny2d_nt1", lambda: synth.random_levels((1, 6, 5), seed=10), 20),
]


def _slice_times(pos, nt, rng, k=6):
    """Times at least 1e-4 away from every point's time (where FP32 and FP64
    could order a point and the slice differently)."""
    ts = np.asarray([p[3] for p in pos.values()]) if pos else np.zeros(0)
    out = []
    while len(out) < k:
        t0 = float(rng.uniform(0.0, max(nt - 1.0, 0.5)))
        if ts.size == 0 or np.min(np.abs(ts - t0)) > 1e-4:
            out.append(t0)
    return out


@pytest.mark.parametrize("name,make,shift", CASES, ids=[c[0] for c in CASES])
def test_trajectories_and_slices_match_oracle(F, name, make, shift):
    f = make()
    ref = cp.track(f, shift=shift)
    trajs = cp.trajectories(ref["grid"], ref["face_id"], ref["label"])
    with F.Plan(f.shape, F.make_params(quant_shift=shift)) as plan:
        plan.execute(torch.from_numpy(f).cuda())
        compare_full(plan.download(), ref)
        off, pts, closed = plan.trajectories()
        assert len(off) == len(trajs) + 1
        for i, (order, cl) in enumerate(trajs):
            got = pts["face_id"][off[i]:off[i + 1]].tolist()
            assert got == order, f"trajectory {i}"
            assert bool(closed[i]) == cl
            assert np.all(pts["label"][off[i]:off[i + 1]] == min(order))
        pos = cp.positions(ref)
        rng = np.random.default_rng(len(name))
        for t0 in _slice_times(pos, f.shape[0], rng):
            want = cp.slice_trajectories(trajs, pos, t0)
            got = plan.slice(t0)
            assert len(got) == len(want), t0
            for g, w in zip(got, want):
                assert (int(g["label"]), int(g["face_a"]), int(g["face_b"])) == w[:3]
                assert np.max(np.abs(g["pos"] - np.asarray(w[3]))) <= OFF_TOL
        if name.startswith("minimum"):
            assert len(trajs) == 1 and not closed[0]


@pytest.mark.parametrize("name,make,shift", [CASES[1], CASES[3], CASES[5], CASES[8]], ids=[CASES[i][0] for i in (1, 3, 5, 8)])
@pytest.mark.parametrize("flt", [
    dict(min_duration=1.45), dict(min_points=4), dict(drop_loops=True), dict(smooth_half_window=2),
    dict(min_duration=0.55, drop_loops=True, smooth_half_window=1),
])
def test_filtered_trajectories_match_oracle(F, name, make, shift, flt):
    f = make()
    ref = cp.track(f, shift=shift)
    trajs = cp.trajectories(ref["grid"], ref["face_id"], ref["label"])
    pos = cp.positions(ref)
    morse = dict(zip(ref["face_id"].tolist(), ref["morse"].tolist()))
    want = cp.filter_trajectories(trajs, pos, morse, min_duration=flt.get("min_duration", 0.0),
                                  min_points=flt.get("min_points", 0), drop_loops=flt.get("drop_loops", False),
                                  half_window=flt.get("smooth_half_window", 0))
    with F.Plan(f.shape, F.make_params(quant_shift=shift)) as plan:
        plan.execute(torch.from_numpy(f).cuda())
        off, pts, closed = plan.trajectories(**flt)
    assert len(off) == len(want) + 1
    for i, (order, cl, types) in enumerate(want):
        assert pts["face_id"][off[i]:off[i + 1]].tolist() == order
        assert pts["morse_index"][off[i]:off[i + 1]].tolist() == types
        assert bool(closed[i]) == cl
