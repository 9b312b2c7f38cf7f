"""GPU isovolume tracking (Sec. 6.1; Algorithm 1, right column) against the
CPU oracle, through the C ABI: intersected edge set, piece labels, base
vertices and ordinal flags equal; crossing points within 1e-5 of an edge
length (FP32 location against the FP64 oracle)."""
import numpy as np
import pytest

from oracle import iso
from paper_2011_08697_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2011_08697_gb300 import build, ftk
    build.build()
    ftk.lib()
    return ftk


def compare(got, ref):
    assert np.array_equal(got["edge_id"], ref["edge_id"]), "intersected edges differ"
    assert np.array_equal(got["label"], ref["label"]), "piece labels differ"
    assert np.array_equal(got["base"].astype(np.int64), ref["base"]), "base vertices differ"
    assert np.array_equal(got["ordinal"].astype(bool), ref["ordinal"]), "ordinal flags differ"
    if len(got):
        err = float(np.max(np.abs(got["off"].astype(np.float64) - ref["off"])))
        assert err <= TOL, f"crossing error {err}"


def track(F, f, c):
    x = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    return F.ftk_track_iso3d(x, c) if f.ndim == 4 else F.ftk_track_iso2d(x, c)


def plane(alpha, dims, nt):
    shape = (nt,) + tuple(reversed(dims))
    t = np.arange(nt, dtype=np.float64).reshape((nt,) + (1,) * len(dims))
    x = np.arange(dims[0], dtype=np.float64).reshape((1,) * len(dims) + (dims[0],))
    return (x - alpha * t + np.zeros(shape)).astype(np.float32)


def noise(shape, seed):
    return np.random.default_rng(seed).normal(size=shape).astype(np.float32)


CASES = {
    "plane3d_21x21x21x12_a0.875": (lambda: plane(0.875, (21, 21, 21), 12), 0.0),
    "plane3d_21x21x21x12_a0.9": (lambda: plane(0.9, (21, 21, 21), 12), 0.0),
    "line2d_17x17x9": (lambda: plane(0.625, (17, 17), 9), 0.0),
    "levels2d_9x31x33": (lambda: synth.random_levels((9, 31, 33), seed=1), 0.0),
    "levels3d_5x9x10x37": (lambda: synth.random_levels((5, 9, 10, 37), seed=2), 0.0),
    "levels3d_4x7x6x64": (lambda: synth.random_levels((4, 7, 6, 64), seed=3), 1.0),
    "noise2d_6x40x100": (lambda: noise((6, 40, 100), 4), 0.1),
    "noise3d_4x12x11x65": (lambda: noise((4, 12, 11, 65), 5), -0.3),
    "blobs3d_40x36x33x5": (lambda: synth.gaussian_blobs((33, 36, 40), 5, nblobs=6, seed=6), 0.25),
    "nt1_3d_1x8x9x40": (lambda: noise((1, 8, 9, 40), 7), 0.0),
    "nt1_2d_1x20x30": (lambda: noise((1, 20, 30), 8), 0.0),
    "thin2d_5x2x2": (lambda: noise((5, 2, 2), 9), 0.0),
    "thin3d_3x2x2x2": (lambda: noise((3, 2, 2, 2), 10), 0.0),
    "empty_above": (lambda: np.ones((3, 6, 7, 8), np.float32), 0.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_parity(F, name):
    make, c = CASES[name]
    f = make()
    compare(track(F, f, c), iso.track_iso(f, c))


def _two_spheres(sep, n=24, nt=6):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    out = np.zeros((nt, n, n, n), dtype=np.float32)
    for t in range(nt):
        a, b = n / 2 - sep(t) / 2, n / 2 + sep(t) / 2
        da = np.sqrt((x - a) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2)
        db = np.sqrt((x - b) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2)
        out[t] = np.minimum(da, db)
    return out


def test_pieces_split_and_merge(F):
    apart = _two_spheres(lambda t: 14.0)
    got = track(F, apart, 4.0)
    compare(got, iso.track_iso(apart, 4.0))
    assert len(np.unique(got["label"])) == 2
    meet = _two_spheres(lambda t: 14.0 - 2.0 * t)
    got = track(F, meet, 4.0)
    compare(got, iso.track_iso(meet, 4.0))
    assert len(np.unique(got["label"])) == 1


def test_plan_reuse_host_input_and_growth(F):
    # 2D noise: about 9e5 intersected edges, far beyond the first capacity
    f = noise((4, 256, 256), 11)
    plan = F.IsoPlan(f.shape)
    for c in (0.0, 0.7):
        plan.execute(torch.from_numpy(f).cuda(), c)
        ref = iso.track_iso(f, c)
        assert plan.count() == len(ref["edge_id"])
        compare(plan.download(), ref)
    host = f.copy()
    plan.execute(host, -0.4)         # host input, copied before execute returns
    host[:] = 9.0
    compare(plan.download(), iso.track_iso(f, -0.4))
    buf = np.zeros(plan.count() + 5, dtype=F.ISO_DTYPE)
    compare(plan.download_into(buf), iso.track_iso(f, -0.4))
    plan.close()


def test_errors(F):
    f = noise((3, 6, 7), 12)
    with pytest.raises(F.FtkError) as e:
        F.ftk_track_iso2d(torch.from_numpy(f).cuda(), float("nan"))
    assert e.value.status == 1
    bad = f.copy()
    bad[1, 2, 3] = np.inf
    with pytest.raises(F.FtkError) as e:
        F.ftk_track_iso2d(torch.from_numpy(bad).cuda(), 0.0)
    assert e.value.status == 2
    with pytest.raises(F.FtkError) as e:
        F.ftk_track_iso2d(torch.from_numpy(np.zeros((3, 1, 7), np.float32)).cuda(), 0.0)
    assert e.value.status == 1


def test_full_size_blobs3d(F):
    """The 128^3 x 16 blob workload at isovalue 0.25, compared in full."""
    f = synth.gaussian_blobs((128, 128, 128), 16, nblobs=32, seed=0)
    compare(track(F, f, 0.25), iso.track_iso(f, 0.25))
