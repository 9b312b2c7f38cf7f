"""In-situ streams: pushing one slice at a time yields, delta by delta, the
faces of the whole-field result (ordinal faces of slice k and interval faces
of slab [k-1, k] at push k) with the oracle's provisional labels, and closing
yields the whole-field result.  Streams give the same results alone and
mixed with other streams pushing concurrently."""
import threading

import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

from parity_util import compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_stream(F, f, device=True, server=None):
    s = F.Stream(f.shape[1:], server=server)
    deltas = []
    for k in range(f.shape[0]):
        sl = torch.from_numpy(np.ascontiguousarray(f[k]))
        deltas.append(s.push(sl.cuda() if device else sl))
    final = s.close()
    return deltas, final


@pytest.mark.parametrize("make", [
    lambda: synth.spiral_woven(40, 7, sigma=0.02, seed=2),
    lambda: synth.random_levels((5, 13, 22), seed=6),
    lambda: synth.random_levels((4, 5, 6, 7), seed=8),
    lambda: synth.gaussian_blobs((36, 20), 1, nblobs=8, seed=3, sigma_range=(2.0, 5.0)),
])
def test_stream_deltas_match_oracle(make):
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    f = make()
    ref = cp.track(f)
    g = ref["grid"]
    ids = [int(x) for x in ref["face_id"]]
    deltas, final = _run_stream(F, f, device=True)
    compare_full(final, ref)
    seen = []
    for k, d in enumerate(deltas):
        want = sorted(fid for fid in ids if cp.stream_push_index(g, fid) == k)
        assert sorted(d["face_id"].tolist()) == want, k
        prov = cp.stream_labels(g, ids, k)
        for fid, lab in zip(d["face_id"].tolist(), d["label"].tolist()):
            assert lab == prov[fid]
        seen += d["face_id"].tolist()
    assert sorted(seen) == ids
    # host slices give the same deltas
    deltas_h, final_h = _run_stream(F, f, device=False)
    for a, b in zip(deltas, deltas_h):
        assert np.array_equal(np.sort(a["face_id"]), np.sort(b["face_id"]))
    compare_full(final_h, ref)


def test_streams_alone_equal_mixed_and_admission():
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    fields = [synth.gaussian_blobs((48 + 8 * i, 40), 6, nblobs=10, seed=20 + i, sigma_range=(2.0, 6.0))
              for i in range(4)]
    alone = [_run_stream(F, f)[1] for f in fields]
    srv = F.Server(1 << 34)
    results = [None] * len(fields)

    def worker(i):
        results[i] = _run_stream(F, fields[i], server=srv)[1]

    th = [threading.Thread(target=worker, args=(i,)) for i in range(len(fields))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for a, m in zip(alone, results):
        assert np.array_equal(a["face_id"], m["face_id"])
        assert np.array_equal(a["label"], m["label"])
        assert np.array_equal(a["morse_index"], m["morse_index"])
    assert srv.used() == 0
    # a budget below one stream's footprint refuses admission
    tiny = F.Server(1 << 10)
    with pytest.raises(F.FtkError) as e:
        F.Stream((40, 48), server=tiny)
    assert e.value.status == 6
    tiny.close()
    srv.close()
