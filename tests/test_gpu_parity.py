"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact punctured-face set, Morse index, ordinal flag and trajectory labels;
FP32 locations within 1e-5 of a grid spacing of the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

from parity_util import OFF_TOL, WindowOracle, compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2011_08697_gb300 import build, ftk
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ftk


def _gpu(F, f, shift=20, host=False, max_punctures=0):
    p = F.make_params(quant_shift=shift, max_punctures=max_punctures)
    arg = f if host else torch.from_numpy(f).cuda()
    if f.ndim == 3:
        return F.ftk_track_cp2d(arg, p)
    return F.ftk_track_cp3d(arg, p)


CASES = [
    ("spiral_32x32x10", lambda: synth.spiral_woven(32, 10), 20),
    ("spiral_noisy_61x47x9", lambda: synth.spiral_woven(61, 9, sigma=0.02, seed=3, ny=47), 20),
    ("levels2d_37x23x5", lambda: synth.random_levels((5, 23, 37), seed=1), 20),
    ("levels2d_5lvl_19x30x4", lambda: synth.random_levels((4, 30, 19), levels=(-1, -.5, 0, .5, 1), seed=2), 20),
    ("levels3d_11x9x7x4", lambda: synth.random_levels((4, 7, 9, 11), seed=4), 20),
    ("levels3d_6x13x5x3", lambda: synth.random_levels((3, 5, 13, 6), levels=(-1, -.5, 0, .5, 1), seed=5), 20),
    ("minimum2d", lambda: synth.moving_minimum(21, 8, (10, 10), (0.5, 0.5), 2), 17),
    ("minimum3d", lambda: synth.moving_minimum(13, 4, (6, 6, 6), (0.25, -0.5, 0.75), 3), 17),
    ("blobs3d_40x36x33x5", lambda: synth.gaussian_blobs((40, 36, 33), 5, nblobs=12, seed=7,
                                                         sigma_range=(2.0, 6.0)), 20),
    ("blobs2d_301x45x6", lambda: synth.gaussian_blobs((301, 45), 6, nblobs=20, seed=8,
                                                       sigma_range=(2.0, 8.0)), 20),
    ("tiny2d_2x2x2", lambda: synth.random_levels((2, 2, 2), seed=9), 20),
    ("tiny2d_nt1", lambda: synth.random_levels((1, 6, 5), seed=10), 20),
    ("tiny3d_2x2x2x2", lambda: synth.random_levels((2, 2, 2, 2), seed=11), 20),
    ("thin2d_2x50x7", lambda: synth.random_levels((7, 50, 2), seed=12), 20),
    ("zero_field", lambda: np.zeros((3, 8, 9), np.float32), 20),
    # shapes taking the streaming 2D kernel (nx % 4 == 0)
    ("stream_levels_36x23x5", lambda: synth.random_levels((5, 23, 36), seed=13), 20),
    ("stream_levels_4x40x3", lambda: synth.random_levels((3, 40, 4), seed=14), 20),
    ("stream_levels5_8x17x2", lambda: synth.random_levels((2, 17, 8), levels=(-1, -.5, 0, .5, 1), seed=15), 20),
    ("stream_zero_12x10x3", lambda: np.zeros((3, 10, 12), np.float32), 20),
    ("stream_nt1_64x48", lambda: synth.spiral_woven(64, 1, ny=48), 20),
    ("stream_wide_values", lambda: (synth.spiral_woven(64, 6, sigma=0.01, seed=5, ny=48) * 10.0), 20),
    ("stream_blobs_256x100x40", lambda: synth.gaussian_blobs((256, 100), 40, nblobs=30, seed=16,
                                                              sigma_range=(2.0, 9.0)), 20),
    ("stream_levels_20x37x7", lambda: synth.random_levels((7, 37, 20), levels=(-1, -.5, 0, .5, 1), seed=17), 20),
    ("stream_noisy_128x33x12", lambda: synth.spiral_woven(128, 12, sigma=0.05, seed=6, ny=33), 20),
    ("stream_wide_2900x4x3", lambda: synth.random_levels((3, 4, 2900), seed=35), 20),
    ("stream_wide_4093x5x2", lambda: synth.random_levels((2, 5, 4093), levels=(-1, -.5, 0, .5, 1), seed=38), 20),
    # shapes taking the streaming 3D kernel (rows padded to 4 floats, <= 1024)
    ("s3_levels_8x9x7x4", lambda: synth.random_levels((4, 7, 9, 8), seed=21), 20),
    ("s3_levels5_12x5x6x3", lambda: synth.random_levels((3, 6, 5, 12), levels=(-1, -.5, 0, .5, 1), seed=22), 20),
    ("s3_tiny_4x2x2x2", lambda: synth.random_levels((2, 2, 2, 4), seed=23), 20),
    ("s3_nt1_16x10x9", lambda: synth.random_levels((1, 9, 10, 16), seed=24), 20),
    ("s3_zero_8x6x5x3", lambda: np.zeros((3, 5, 6, 8), np.float32), 20),
    ("s3_wide_132x4x3x2", lambda: synth.random_levels((2, 3, 4, 132), seed=25), 20),
    ("s3_wide_264x3x3x2", lambda: synth.random_levels((2, 3, 3, 264), seed=26), 20),
    ("s3_wide_600x4x3x2", lambda: synth.random_levels((2, 3, 4, 600), seed=30), 20),
    ("s3_wide_1021x3x2x2", lambda: synth.random_levels((2, 2, 3, 1021), levels=(-1, -.5, 0, .5, 1), seed=31), 20),
    ("s3_blobs_1024x9x4x3", lambda: synth.gaussian_blobs((1024, 9, 4), 3, nblobs=40, seed=32,
                                                          sigma_range=(2.0, 6.0)), 20),
    # wider than the streaming kernels: the tiled kernel on windows of the row
    ("tile3_wide_1030x3x3x2", lambda: synth.random_levels((2, 3, 3, 1030), seed=33), 20),
    ("tile3_wide_1600x2x2x2", lambda: synth.random_levels((2, 2, 2, 1600), levels=(-1, -.5, 0, .5, 1), seed=34), 20),
    ("tile2_wide_6000x3x2", lambda: synth.random_levels((2, 3, 6000), levels=(-1, -.5, 0, .5, 1), seed=36), 20),
    ("tile2_blobs_4100x12x4", lambda: synth.gaussian_blobs((4100, 12), 4, nblobs=60, seed=37,
                                                            sigma_range=(2.0, 6.0)), 20),
    ("s3_levels5_20x17x9x3", lambda: synth.random_levels((3, 9, 17, 20), levels=(-1, -.5, 0, .5, 1), seed=27), 20),
    ("s3_blobs_36x40x20x6", lambda: synth.gaussian_blobs((36, 40, 20), 6, nblobs=16, seed=28,
                                                          sigma_range=(2.0, 6.0)), 20),
    ("s3_wide_values", lambda: synth.gaussian_blobs((24, 20, 18), 4, nblobs=10, seed=29,
                                                     sigma_range=(2.0, 5.0)) * 10.0, 20),
]


@pytest.mark.parametrize("name,make,shift", CASES, ids=[c[0] for c in CASES])
def test_parity_small(F, name, make, shift):
    f = make()
    ref = cp.track(f, shift=shift)
    got = _gpu(F, f, shift)
    compare_full(got, ref)


def test_host_pointer_and_capacity_growth(F):
    f = synth.random_levels((5, 23, 37), seed=1)
    ref = cp.track(f)
    compare_full(_gpu(F, f, host=True), ref)
    # a tiny initial capacity forces the overflow / re-run path
    compare_full(_gpu(F, f, max_punctures=16), ref)
    f3 = synth.random_levels((4, 7, 9, 11), seed=4)
    compare_full(_gpu(F, f3, host=True, max_punctures=8), cp.track(f3))
    # a device pointer that is not 16-byte aligned (rows are copied by TMA)
    f2 = synth.random_levels((5, 23, 36), seed=13)
    buf = torch.empty(f2.size + 1, dtype=torch.float32, device="cuda")
    x = buf[1:].view(f2.shape)
    x.copy_(torch.from_numpy(f2))
    assert x.data_ptr() % 16 != 0
    compare_full(F.ftk_track_cp2d(x, F.make_params()), cp.track(f2))


def test_plan_reuse_and_device_view(F):
    f = synth.spiral_woven(32, 10)
    ref = cp.track(f)
    with F.Plan(f.shape, F.make_params(flags=F.FTK_FLAG_STAGE_TIMES)) as plan:
        x = torch.from_numpy(f).cuda()
        for _ in range(3):
            plan.execute(x)
            compare_full(plan.download(), ref)
        v = plan.device_view()
        assert v.count == len(ref["face_id"])
        st = plan.stage_times()
        assert len(st) == 5 and all(s >= 0 for s in st)


def test_range_errors(F):
    f = synth.spiral_woven(16, 3)
    f[1, 3, 4] = 1.0e6          # 1e6 * 2^20 > 2^28
    with pytest.raises(F.FtkError) as e:
        _gpu(F, f)
    assert e.value.status == 2
    f[1, 3, 4] = np.nan
    with pytest.raises(F.FtkError) as e:
        _gpu(F, f)
    assert e.value.status == 2
    # a smaller quantisation shift brings the same value back in range
    f[1, 3, 4] = 100.0
    compare_full(_gpu(F, f, shift=12), cp.track(f, shift=12))


@pytest.mark.parametrize("shape,maker", [
    ((16, 256, 256), "spiral"),
    ((6, 48, 48, 48), "blobs3d"),
])
def test_parity_medium_full(F, shape, maker):
    """Full element-by-element parity at sizes spanning many detect tiles and
    time chunks, with ragged tails."""
    if maker == "spiral":
        f = synth.spiral_woven(shape[2], shape[0], sigma=1e-3, seed=0, ny=shape[1])
    else:
        f = synth.gaussian_blobs(tuple(reversed(shape[1:])), shape[0], nblobs=24, seed=2,
                                 sigma_range=(3.0, 8.0))
    ref = cp.track(f)
    got = _gpu(F, f)
    assert len(got) > 50
    compare_full(got, ref)


def _sampled_full_size(F, f, shift=20, n_punct=1500, n_rand=6000, seed=0):
    got = _gpu(F, f, shift)
    ids = got["face_id"]
    assert len(ids) > 0 and np.all(np.diff(ids) > 0)
    W = WindowOracle(f, shift)
    rng = np.random.default_rng(seed)
    T = W.grid.T
    # 1) sampled punctures: oracle agrees on the verdict, location and type
    pick = rng.choice(len(ids), size=min(n_punct, len(ids)), replace=False)
    for i in pick:
        ex, pun, off, morse = W.face(ids[i])
        assert ex and pun, f"face {ids[i]} punctured on GPU only"
        assert np.max(np.abs(off - got["off"][i])) <= OFF_TOL
        assert morse == got["morse_index"][i]
    # 2) uniformly random faces and 3) every face type at the base vertices of
    # sampled punctures (the near-degenerate neighbourhood)
    nverts = W.grid.nverts
    cand = list(rng.integers(0, nverts * T, size=n_rand))
    for i in pick[:300]:
        g = int(ids[i]) // T
        cand += [g * T + tt for tt in range(T)]
    idset = set(int(x) for x in ids)
    for fid in cand:
        ex, pun, _, _ = W.face(int(fid), want_type=False)
        assert pun == (int(fid) in idset), f"verdict differs on face {fid}"
    # 4) linking: the oracle's partners of sampled punctures carry the same
    # GPU label; every label is the smallest id of its group
    lab = dict(zip(ids.tolist(), got["label"].tolist()))
    for i in pick[:400]:
        for hit in W.partners(int(ids[i])):
            assert len(hit) == 1
            assert lab[hit[0]] == lab[int(ids[i])]
    labels = got["label"]
    uniq, first = np.unique(labels, return_index=True)
    assert np.all(np.isin(uniq, ids))
    for L_ in uniq[: 2000]:
        assert lab[int(L_)] == int(L_)
    assert np.all(labels <= ids)
    return got


def test_full_size_2d_spiral_noisy(F):
    """1024^2 x 64 spiral woven + N(0, 1e-3^2): the plain single-field 2D workload."""
    f = synth.spiral_woven(1024, 64, sigma=1e-3, seed=0)
    got = _sampled_full_size(F, f)
    assert len(np.unique(got["label"])) > 10


def test_full_size_3d_blobs(F):
    """128^3 x 16, 32 moving Gaussian blobs: the 3D pentatope-mesh workload."""
    f = synth.gaussian_blobs((128, 128, 128), 16, nblobs=32, seed=0)
    got = _sampled_full_size(F, f, n_punct=800, n_rand=3000)
    assert set(np.unique(got["morse_index"])) <= {-1, 0, 1, 2, 3}
