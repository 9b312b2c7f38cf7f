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


def test_batched_push_equals_alone():
    """ftk_streams_push (one slice for each of several streams per call, their
    device work overlapping) gives every stream the deltas and final result
    it gets pushed alone, and the oracle's."""
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    fields = [synth.gaussian_blobs((48 + 8 * i, 40 + 4 * i), 7, nblobs=10, seed=40 + i, sigma_range=(2.0, 6.0))
              for i in range(3)]
    fields.append(synth.random_levels((7, 21, 30), seed=44))
    alone = [_run_stream(F, f) for f in fields]
    srv = F.Server(1 << 34)
    streams = [F.Stream(f.shape[1:], server=srv) for f in fields]
    deltas = [[] for _ in fields]
    for k in range(fields[0].shape[0]):
        xs = [torch.from_numpy(np.ascontiguousarray(f[k])).cuda() for f in fields]
        for i, d in enumerate(F.ftk_streams_push(streams, xs)):
            deltas[i].append(d)
    finals = [s.close() for s in streams]
    for i, f in enumerate(fields):
        ref_d, ref_final = alone[i]
        for a, b in zip(deltas[i], ref_d):
            assert np.array_equal(a["face_id"], b["face_id"]) and np.array_equal(a["label"], b["label"])
        compare_full(finals[i], cp.track(f))
        assert np.array_equal(finals[i]["face_id"], ref_final["face_id"])
    assert srv.used() == 0
    srv.close()


def test_admission_waits_for_a_closing_stream():
    """A stream that does not fit the budget waits (first come, first served)
    and is admitted once a closing stream frees its footprint; its results
    are the same as alone.  A wait that runs out refuses with FTK_ERR_BUSY."""
    import time
    from paper_2011_08697_gb300 import build, ftk as F
    build.build()
    fa = synth.gaussian_blobs((48, 40), 6, nblobs=10, seed=50, sigma_range=(2.0, 6.0))
    fb = synth.gaussian_blobs((48, 40), 6, nblobs=10, seed=51, sigma_range=(2.0, 6.0))
    fp = F.ftk_stream_footprint((40, 48))
    srv = F.Server(fp + fp // 2)            # room for one stream, not two
    a = F.Stream((40, 48), server=srv)
    assert srv.used() == fp
    with pytest.raises(F.FtkError) as e:    # no waiting: refused at once
        F.Stream((40, 48), server=srv)
    assert e.value.status == 6
    t0 = time.perf_counter()
    with pytest.raises(F.FtkError) as e:    # a bounded wait that runs out
        F.Stream((40, 48), server=srv, wait_ms=200)
    assert e.value.status == 6 and time.perf_counter() - t0 >= 0.15
    got = {}

    def opener():
        s = F.Stream((40, 48), server=srv, wait_ms=60_000)
        got["admitted_at"] = time.perf_counter()
        got["res"] = [s.push(torch.from_numpy(np.ascontiguousarray(fb[k])).cuda()) for k in range(fb.shape[0])]
        got["final"] = s.close()

    th = threading.Thread(target=opener)
    th.start()
    for k in range(fa.shape[0]):            # a keeps running while b waits
        a.push(torch.from_numpy(np.ascontiguousarray(fa[k])).cuda())
    time.sleep(0.3)
    assert "admitted_at" not in got
    t_close = time.perf_counter()
    fa_final = a.close()
    th.join(timeout=120)
    assert not th.is_alive()
    assert got["admitted_at"] >= t_close
    compare_full(got["final"], cp.track(fb))
    compare_full(fa_final, cp.track(fa))
    assert srv.used() == 0
    srv.close()
