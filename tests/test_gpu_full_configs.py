"""Bit-exact parity on the full workloads, element by element.

Every punctured face, its Morse index, ordinal flag, base vertex and
trajectory label from the CUDA path (through the C ABI) must equal the
oracle's, and every FP32 in-cell offset must lie within 1e-5 of a grid
spacing of the oracle's FP64 location:

* spiral woven 1024^2 x 64 with N(0, 1e-3^2) noise (plain 2D path);
* 32 moving Gaussian blobs on 128^3 x 16 (plain 3D path);
* 256 independent blob fields, N log-uniform in 64..512, 8..32 slices, run
  as one batch (graph-captured after the first execute);
* one in-situ stream of a 1235^2 blob field pushed one slice at a time for
  48 slices: every delta against the oracle's faces of that push and its
  provisional labels, and the final result against the whole-field oracle.

The oracle runs on all host cores (``cp.track_parallel`` / ``cp.track_many``,
spawned processes: safe next to the CUDA context).
"""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

from parity_util import compare_full

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2011_08697_gb300 import build, ftk
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ftk


def test_full_spiral2d_1024x1024x64(F):
    f = synth.spiral_woven(1024, 64, sigma=1e-3, seed=0)
    got = F.ftk_track_cp2d(torch.from_numpy(f).cuda())
    ref = cp.track_parallel(f)
    assert len(ref["face_id"]) > 1_000_000
    compare_full(got, ref)


def test_full_blobs3d_128x128x128x16(F):
    f = synth.gaussian_blobs((128, 128, 128), 16, nblobs=32, seed=0)
    got = F.ftk_track_cp3d(torch.from_numpy(f).cuda())
    ref = cp.track_parallel(f)
    assert len(ref["face_id"]) > 1000
    compare_full(got, ref)


def test_full_batch_256_fields(F):
    specs = synth.batch_fields(256, materialise=False)
    dev = torch.device("cuda")
    xs = [synth.blob_slices_torch(bs, 0, nt, dev) for (_, _, nt, _, bs) in specs]
    torch.cuda.synchronize()
    fields = [x.cpu().numpy() for x in xs]
    with F.Batch([f.shape for f in fields], F.make_params(flags=F.FTK_FLAG_AUTOTUNE)) as b:
        b.execute(xs)              # first execute: uncaptured, autotuned
        b.download()
        b.execute(xs)              # graph replay
        got = b.download()
    refs = cp.track_many(fields)
    for i, (g, r) in enumerate(zip(got, refs)):
        try:
            compare_full(g, r)
        except AssertionError as e:
            raise AssertionError(f"field {i} {fields[i].shape}: {e}") from None
    assert sum(len(r["face_id"]) for r in refs) > 1000


def test_full_stream_1235x1235x48(F):
    n, bs = synth.stream_specs(32)[16]
    assert n >= 1024
    nt = 48
    f = np.stack([synth.blob_slice(bs, k) for k in range(nt)])
    ref = cp.track_parallel(f)
    ids = [int(x) for x in ref["face_id"]]
    g = ref["grid"]
    s = F.Stream((n, n))
    deltas = [s.push(torch.from_numpy(np.ascontiguousarray(f[k])).cuda()) for k in range(nt)]
    final = s.close()
    compare_full(final, ref)
    by_push = {}
    for fid in ids:
        by_push.setdefault(cp.stream_push_index(g, fid), []).append(fid)
    seen = 0
    for k, d in enumerate(deltas):
        want = sorted(by_push.get(k, []))
        assert sorted(d["face_id"].tolist()) == want, f"push {k}"
        prov = cp.stream_labels(g, [x for x in ids if cp.stream_push_index(g, x) <= k], k)
        for fid, lab in zip(d["face_id"].tolist(), d["label"].tolist()):
            assert lab == prov[fid], f"push {k} face {fid}"
        seen += len(d)
    assert seen == len(ids)
