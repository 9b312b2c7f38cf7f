"""Helpers shared by the GPU parity tests: run the oracle, compare results,
and check single faces of a full-size field against the oracle through small
windows (so no full-field oracle arrays are needed)."""
from __future__ import annotations

import numpy as np

from oracle import cp

# FP32 location vs the FP64 oracle, in in-cell (grid-spacing) units
OFF_TOL = 1e-5


def oracle_result(f, shift=20):
    r = cp.track(f, shift=shift)
    return r


def compare_full(gpu, ref, tol=OFF_TOL):
    """Bit-exact punctured set, Morse index, ordinal flag, base and labels;
    offsets within tol."""
    ids = gpu["face_id"]
    assert np.all(np.diff(ids) > 0), "GPU result not sorted by face id"
    assert np.array_equal(ids, ref["face_id"]), (
        f"punctured sets differ: gpu {len(ids)} oracle {len(ref['face_id'])}; "
        f"only-gpu {np.setdiff1d(ids, ref['face_id'])[:10]} "
        f"only-oracle {np.setdiff1d(ref['face_id'], ids)[:10]}")
    assert np.array_equal(gpu["morse_index"], ref["morse"])
    assert np.array_equal(gpu["ordinal"], ref["ordinal"])
    assert np.array_equal(gpu["base"], ref["base"])
    assert np.array_equal(gpu["label"], ref["label"])
    if len(ids):
        err = np.max(np.abs(gpu["off"].astype(np.float64) - ref["off"]))
        assert err <= tol, f"max offset error {err}"
        return float(err)
    return 0.0


class WindowOracle:
    """Oracle verdicts for individual faces of a large field, computed on a
    window of +-3 cells around the face (enough for gradients and Hessians:
    window edges that are not grid edges stay >= 2 cells from every vertex
    used)."""

    def __init__(self, f, shift=20):
        self.f = f
        self.shift = shift
        self.n = f.ndim - 1
        self.nt = f.shape[0]
        self.dims = tuple(reversed(f.shape[1:]))
        self.grid = cp.Grid(self.dims, self.nt)

    def _window(self, base):
        n = self.n
        lo, hi = [], []
        for a in range(n):
            lo.append(max(0, base[a] - 3))
            hi.append(min(self.dims[a], base[a] + 5))
        t0, t1 = base[n], min(self.nt, base[n] + 2)
        sl = [slice(t0, t1)] + [slice(lo[a], hi[a]) for a in reversed(range(n))]
        w = self.f[tuple(sl)]
        F = cp.quantise(w, self.shift)
        G = cp.gradient(F, n)
        H = cp.hessian(G, n)
        return lo, t0, G, H

    def face(self, fid, want_type=True):
        """(exists, punctured, off[4] or None, morse or None)."""
        g = self.grid
        base, chain = g.decode_face(int(fid))
        if not g.face_exists(base, chain):
            return False, False, None, None
        lo, t0, G, H = self._window(base)
        verts = g.simplex_vertices(base, chain)
        n = self.n

        def loc(v):
            return (v[n] - t0,) + tuple(v[a] - lo[a] for a in reversed(range(n)))

        V = [[int(x) for x in G[loc(v)]] for v in verts]
        if not cp.face_punctured(V):
            return True, False, None, None
        mu, D = cp.barycentric(V)
        ms = [0] + list(chain)
        off = np.zeros(4)
        for a in range(g.d):
            off[a if a < n else 3] = sum(float(mu[k]) for k in range(n + 1) if (ms[k] >> a) & 1)
        morse = cp.classify(D, [H[loc(v)] for v in verts]) if want_type else None
        return True, True, off, morse

    def partners(self, fid):
        """Punctured partner faces of fid, one per coface (oracle verdicts)."""
        g = self.grid
        base, chain = g.decode_face(int(fid))
        out = []
        for cb, cc in g.cofaces(base, chain):
            hit = []
            for sb, sc in g.cell_sides(cb, cc):
                sid = g.face_id(sb, sc)
                if sid == fid:
                    continue
                if self.face(sid, want_type=False)[1]:
                    hit.append(sid)
            out.append(hit)
        return out
