"""Pins of the oracle's vector-field tracking (paper Sec. 4.1: critical
points of a vector field v are its zeros; sources, sinks and saddles from
the eigenvalues of the Jacobian).

* Linear fields v = A (x - c0 - d t): the PL interpolation of a linear field
  is exact and central differences give A exactly, so there is one
  trajectory, the line c0 + d t (its slice at any t is that point), and its
  type is fixed by the eigenvalues of A, computed here independently.
* A gradient field handed over as a vector field, v = G / 2^S with G the
  oracle's integer gradient of a scalar field, quantises back to G: the
  punctured faces, trajectories and locations equal the scalar tracking's.
* Degenerate {-1, 0, 1} vector fields keep the 0-or-2 pairing invariant
  (linking raises otherwise).
"""
import numpy as np
import pytest

from oracle import cp
from paper_2011_08697_gb300 import synth


def _eig_type(A):
    ev = np.linalg.eigvals(np.asarray(A, dtype=np.float64))
    if np.any(np.abs(ev.real) < 1e-12):
        return -1
    return int(np.sum(ev.real < 0))


@pytest.mark.parametrize("A", [
    [[1, 0], [0, 1]], [[-1, 0], [0, -1]], [[1, 0], [0, -1]], [[-1, -2], [2, -1]],
    [[1, 2], [-2, 1]], [[0, -1], [1, 0]], [[0.5, 1], [0, 0.25]], [[-0.75, 0.5], [0.25, 0.5]],
])
def test_linear_field_single_line_and_type(A):
    c0, d, nt = (8.0, 7.5), (0.25, 0.5), 6
    v = synth.linear_vector_field(17, nt, A, c0, d)
    r = cp.track_vec(v, shift=16)
    trajs = cp.trajectories(r["grid"], r["face_id"], r["label"])
    assert len(trajs) == 1 and not trajs[0][1]
    assert set(r["morse"].tolist()) == {_eig_type(A)}
    pos = cp.positions(r)
    for t0 in (0.3, 1.0, 2.7, 4.9):
        pts = cp.slice_trajectories(trajs, pos, t0)
        assert len(pts) == 1
        assert np.allclose(pts[0][3][:2], (c0[0] + d[0] * t0, c0[1] + d[1] * t0), atol=1e-9)


@pytest.mark.parametrize("make", [
    lambda: synth.spiral_woven(40, 6, sigma=0.02, seed=2),
    lambda: synth.gaussian_blobs((30, 26), 5, nblobs=8, seed=3, sigma_range=(2.0, 5.0)),
])
def test_gradient_field_as_vectors_equals_scalar_tracking(make):
    f = make()
    ref = cp.track(f)
    G = cp.gradient(cp.quantise(f), 2)
    assert np.max(np.abs(G)) < (1 << 24)                 # exact as float32 after the scale
    v = (G.astype(np.float64) / float(1 << 20)).astype(np.float32)
    got = cp.track_vec(v)
    for k in ("face_id", "label", "ordinal", "base"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.max(np.abs(got["off"] - ref["off"])) == 0.0


def test_degenerate_vector_field_pairs():
    rng = np.random.default_rng(5)
    v = rng.integers(-1, 2, size=(4, 11, 13, 2)).astype(np.float32)
    r = cp.track_vec(v)                                  # raises on a broken pairing
    assert len(r["face_id"]) > 0 and set(r["morse"].tolist()) <= {-1, 0, 1, 2}
