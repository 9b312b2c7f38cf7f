"""The seeded generators: the device-side blob generator used by the batch
and serving benchmarks follows the same law as the NumPy one."""
import numpy as np
import pytest

from paper_2011_08697_gb300 import synth


def test_torch_blob_slices_match_numpy():
    torch = pytest.importorskip("torch")
    bs = synth.blob_set((70, 50), 12, seed=3, sigma_range=(2.0, 6.0))
    a = np.stack([synth.blob_slice(bs, k) for k in range(5)])
    b = synth.blob_slices_torch(bs, 0, 5, "cpu", chunk=2).numpy()
    assert a.shape == b.shape == (5, 50, 70)
    assert np.max(np.abs(a - b)) <= 1e-6 * max(1.0, float(np.max(np.abs(a))))


def test_batch_and_stream_specs_are_seeded():
    a = synth.batch_fields(8, materialise=False)
    b = synth.batch_fields(8, materialise=False)
    assert [(n, nt) for n, _, nt, _, _ in a] == [(n, nt) for n, _, nt, _, _ in b]
    assert all(64 <= n <= 512 and 8 <= nt <= 32 for n, _, nt, _, _ in a)
    s = synth.stream_specs(32)
    assert all(256 <= n <= 2048 for n, _ in s)
    ev = synth.poisson_arrivals(4, 100.0, 2.0, seed=1)
    assert ev == sorted(ev) and all(0 <= t <= 2.0 for t, _ in ev)
