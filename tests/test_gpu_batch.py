"""Batched tracking (one CUDA graph over many fields) equals the plain
per-field path and the oracle, on fields of uneven size and length."""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

from parity_util import compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields():
    out = []
    # a few small fields the oracle checks in full, of mixed widths (nx % 4 != 0
    # takes the tile kernel, nx % 4 == 0 the streaming kernel), one with nt = 1
    for i, (n, nt) in enumerate([(37, 5), (64, 9), (29, 1), (48, 12), (100, 7), (33, 3)]):
        bs = synth.blob_set((n, n), 12, seed=100 + i, sigma_range=(2.0, 6.0))
        out.append(np.stack([synth.blob_slice(bs, k) for k in range(nt)]))
    out.append(synth.random_levels((4, 21, 36), seed=3))
    return out


def _same(a, b):
    assert np.array_equal(a["face_id"], b["face_id"])
    for k in ("label", "morse_index", "ordinal", "base"):
        assert np.array_equal(a[k], b[k]), k
    if len(a):
        assert float(np.max(np.abs(a["off"] - b["off"]))) <= 1e-6


def test_batch_equals_plain_and_oracle():
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    fields = _fields()
    xs = [torch.from_numpy(f).cuda() for f in fields]
    plain = [F.ftk_track_cp2d(x) for x in xs]
    for f, r in zip(fields, plain):
        compare_full(r, cp.track(f))
    with F.Batch([f.shape for f in fields], F.make_params(flags=F.FTK_FLAG_AUTOTUNE)) as b:
        b.execute(xs)                       # first run: uncaptured, autotuned
        for got, ref in zip(b.download(), plain):
            _same(got, ref)
        for _ in range(2):                  # graph replays
            b.execute(xs)
            assert list(b.counts()) == [len(r) for r in plain]
            for got, ref in zip(b.download(), plain):
                _same(got, ref)
        # new input buffers: the graph is captured again
        xs2 = [x.clone() for x in xs]
        b.execute(xs2)
        for got, ref in zip(b.download(), plain):
            _same(got, ref)


def test_one_shot_batch_and_capacity_growth():
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    fields = _fields()
    xs = [torch.from_numpy(f).cuda() for f in fields]
    plain = [F.ftk_track_cp2d(x) for x in xs]
    got = F.ftk_track_cp2d_batch(xs, F.make_params(max_punctures=8))
    for g, r in zip(got, plain):
        _same(g, r)
