"""Zeros of time-varying 2D vector fields from the CUDA path (through the C
ABI) against the oracle (paper Sec. 4.1: critical points of a vector field
are its zeros; sources, sinks and saddles from the Jacobian's eigenvalues).

Bit-exact punctured-face set, type, ordinal flag, base and labels; FP32
locations within 1e-5 of a grid spacing of the FP64 oracle; the same
polylines and slices as the oracle's.
"""
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


def _gpu(F, v, shift=20, host=False, max_punctures=0):
    p = F.make_params(quant_shift=shift, max_punctures=max_punctures)
    return F.ftk_track_vec2d(v if host else torch.from_numpy(v).cuda(), p)


def _levels(shape, seed, levels=(-1.0, 0.0, 1.0)):
    """Degenerate vector fields: every component drawn from a few levels, so
    zero components and equal vectors are everywhere (SoS decides)."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(levels, np.float32), size=shape).astype(np.float32)


LINEAR = [
    [[1, 0], [0, 1]], [[-1, 0], [0, -1]], [[1, 0], [0, -1]], [[-1, -2], [2, -1]],
    [[1, 2], [-2, 1]], [[0, -1], [1, 0]], [[0.5, 1], [0, 0.25]], [[-0.75, 0.5], [0.25, 0.5]],
]


@pytest.mark.parametrize("A", LINEAR, ids=[f"A{i}" for i in range(len(LINEAR))])
def test_linear_fields(F, A):
    v = synth.linear_vector_field(17, 6, A, (8.0, 7.5), (0.25, 0.5))
    ref = cp.track_vec(v, shift=16)
    got = _gpu(F, v, shift=16)
    compare_full(got, ref)
    assert len(np.unique(got["label"])) == 1


CASES = [
    ("vortex_64x48x8", lambda: synth.vortex_street(64, 48, 8, seed=1), 20),
    ("vortex_odd_61x37x5", lambda: synth.vortex_street(61, 37, 5, seed=2), 20),
    ("vortex_200x80x12", lambda: synth.vortex_street(200, 80, 12, nvort=14, nsrc=8, seed=3), 20),
    ("vortex_512x256x16", lambda: synth.vortex_street(512, 256, 16, nvort=40, nsrc=20, seed=16), 20),
    ("vortex_thin_3x50x4", lambda: synth.vortex_street(3, 50, 4, nvort=2, nsrc=1, seed=4), 20),
    ("vortex_wide_values", lambda: synth.vortex_street(48, 40, 6, seed=5) * 50.0, 16),
    ("levels_19x23x5", lambda: _levels((5, 23, 19, 2), 6), 20),
    ("levels5_16x17x4", lambda: _levels((4, 17, 16, 2), 7, (-1, -.5, 0, .5, 1)), 20),
    ("tiny_2x2x2", lambda: _levels((2, 2, 2, 2), 8), 20),
    ("nt1_9x7", lambda: _levels((1, 7, 9, 2), 9), 20),
    ("zero", lambda: np.zeros((3, 8, 9, 2), np.float32), 20),
    ("noise_33x31x6", lambda: np.random.default_rng(10).standard_normal((6, 31, 33, 2)).astype(np.float32), 20),
    # rows of nx % 4 == 0 vertices (up to 2048) take the streaming kernel in
    # vector mode: a thread of 4 columns, ragged unit rows, 320-thread CTAs
    ("stream_levels_36x21x4", lambda: _levels((4, 21, 36, 2), 13), 20),
    ("stream_levels5_12x35x3", lambda: _levels((3, 35, 12, 2), 14, (-1, -.5, 0, .5, 1)), 20),
    ("stream_vortex_2048x8x3", lambda: synth.vortex_street(2048, 8, 3, nvort=12, nsrc=6, seed=15), 20),
    # rows wider than one detect tile: windows of the row, one row per unit
    ("levels_wide_1700x3x3", lambda: _levels((3, 3, 1700, 2), 11), 20),
    ("vortex_wide_3500x6x4", lambda: synth.vortex_street(3500, 6, 4, nvort=30, nsrc=12, seed=12), 20),
]


@pytest.mark.parametrize("name,make,shift", CASES, ids=[c[0] for c in CASES])
def test_parity(F, name, make, shift):
    v = make()
    compare_full(_gpu(F, v, shift), cp.track_vec(v, shift=shift))


def test_host_input_and_capacity_growth(F):
    v = synth.vortex_street(96, 64, 10, seed=11)
    ref = cp.track_vec(v)
    assert len(ref["face_id"]) > 64
    compare_full(_gpu(F, v, host=True), ref)
    compare_full(_gpu(F, v, max_punctures=16), ref)


def test_unaligned_device_pointer(F):
    """Rows of vectors are copied by bulk copies that need 16-byte aligned
    starts: a view one float into a buffer is tracked from an aligned copy."""
    v = synth.vortex_street(96, 64, 10, seed=11)
    buf = torch.empty(v.size + 1, dtype=torch.float32, device="cuda")
    x = buf[1:].view(v.shape)
    x.copy_(torch.from_numpy(v))
    assert x.data_ptr() % 16 != 0
    compare_full(F.ftk_track_vec2d(x, F.make_params()), cp.track_vec(v))


def test_gradient_as_vectors_equals_scalar(F):
    """The integer gradient of a scalar field handed over as a vector field
    quantises back to itself: same faces, locations and links as the scalar
    tracking (the types differ in kind: Jacobian versus symmetrised
    Hessian)."""
    f = synth.gaussian_blobs((30, 26), 5, nblobs=8, seed=3, sigma_range=(2.0, 5.0))
    G = cp.gradient(cp.quantise(f), 2)
    v = (G.astype(np.float64) / float(1 << 20)).astype(np.float32)
    got = _gpu(F, v)
    sc = F.ftk_track_cp2d(torch.from_numpy(f).cuda(), F.make_params())
    for k in ("face_id", "label", "ordinal", "base"):
        assert np.array_equal(got[k], sc[k]), k
    assert np.max(np.abs(got["off"] - sc["off"])) == 0.0
    compare_full(got, cp.track_vec(v))


def test_range_errors(F):
    v = synth.vortex_street(24, 20, 3, seed=12)
    v[1, 3, 4, 1] = np.nan
    with pytest.raises(F.FtkError) as e:
        _gpu(F, v)
    assert e.value.status == 2
    v[1, 3, 4, 1] = 1.0e6            # 1e6 * 2^20 > 2^28
    with pytest.raises(F.FtkError) as e:
        _gpu(F, v)
    assert e.value.status == 2
    v[1, 3, 4, 1] = 100.0
    compare_full(_gpu(F, v, shift=12), cp.track_vec(v, shift=12))


def test_plan_reuse_trajectories_and_slices(F):
    shape = (9, 40, 56, 2)
    with F.Plan(shape, F.make_params(), vec2d=True) as plan:
        for seed in (13, 14):
            v = synth.vortex_street(56, 40, 9, seed=seed)
            ref = cp.track_vec(v)
            plan.execute(torch.from_numpy(v).cuda())
            compare_full(plan.download(), ref)
            trajs = cp.trajectories(ref["grid"], ref["face_id"], ref["label"])
            off, pts, closed = plan.trajectories()
            assert len(off) == len(trajs) + 1
            for i, (order, cl) in enumerate(trajs):
                assert pts["face_id"][off[i]:off[i + 1]].tolist() == order
                assert bool(closed[i]) == cl
            pos = cp.positions(ref)
            ts = np.asarray([p[3] for p in pos.values()])
            for t0 in (0.37, 2.61, 5.13, 7.77):
                if ts.size and np.min(np.abs(ts - t0)) <= 1e-4:
                    continue
                want = cp.slice_trajectories(trajs, pos, t0)
                got = plan.slice(t0)
                assert len(got) == len(want)
                for g, w in zip(got, want):
                    assert (int(g["label"]), int(g["face_a"]), int(g["face_b"])) == w[:3]
                    assert np.max(np.abs(g["pos"] - np.asarray(w[3]))) <= OFF_TOL
        with pytest.raises(ValueError):
            plan.execute(torch.zeros((9, 40, 56), device="cuda"))


def test_types_cover_sources_sinks_saddles(F):
    v = synth.vortex_street(128, 64, 6, nvort=10, nsrc=8, seed=15)
    got = _gpu(F, v)
    kinds = set(got["morse_index"].tolist())
    assert {0, 1, 2} <= kinds
