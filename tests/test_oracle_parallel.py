"""The oracle spread over host threads and processes computes exactly what
the single-threaded oracle computes (same face ids, locations, types and
labels), and the SoS sign read from the eps^0 coefficient first equals the
full expansion's sign (the definition, Sec. 4.3)."""
import itertools

import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth

FIELDS = [
    lambda: synth.random_levels((5, 13, 22), seed=6),
    lambda: synth.random_levels((4, 5, 6, 7), seed=8),
    lambda: synth.spiral_woven(40, 7, sigma=0.02, seed=2),
    lambda: synth.gaussian_blobs((20, 18, 16), 5, nblobs=8, seed=3, sigma_range=(2.0, 5.0)),
    lambda: synth.random_levels((1, 6, 5), seed=10),
]
KEYS = ("face_id", "base", "off", "morse", "ordinal", "label")


def _same(a, b):
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("make", FIELDS)
def test_threaded_scan_equals_serial(make):
    f = make()
    _same(cp.track(f, threads=4), cp.track(f))


def test_process_pool_equals_serial():
    fields = [m() for m in FIELDS]
    refs = [cp.track(f) for f in fields]
    for f, r in zip(fields[:4], refs):
        _same(cp.track_parallel(f, workers=3), r)
    for got, r in zip(cp.track_many(fields, workers=3), refs):
        _same(got, r)


def test_sos_sign_first_coefficient_equals_expansion():
    for n in (2, 3):
        for vals in itertools.product((-1, 0, 1), repeat=n * n):
            M = np.asarray(vals, dtype=np.int64).reshape(n, n)
            assert cp.sos_det_sign(M) == cp.sos_det_sign_expand(M)
    rng = np.random.default_rng(0)
    for _ in range(3000):
        n = int(rng.integers(2, 4))
        M = rng.integers(-3, 4, size=(n, n)) * (1 << int(rng.integers(0, 28)))
        assert cp.sos_det_sign(M) == cp.sos_det_sign_expand(M)
