"""Pins for the oracle's exact puncture predicate (paper Sec. 4.2-4.3, Eq. 1).

The Simulation-of-Simplicity sign is the sign, for every small enough eps > 0,
of the determinant of the perturbed matrix.  These tests evaluate that
perturbed determinant (and the perturbed Eq. 1 system) at a concrete dyadic
eps with exact rational arithmetic, which is independent of the oracle's
symbolic expansion.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import cp

# With integer entries |m| <= 2 and n <= 3 the eps-polynomial of a determinant
# has sum of |coefficients| <= n! * 3^n = 162 < 2^8, so at eps = 2^-8 its sign
# is the sign of its lowest-order nonzero term, i.e. the SoS sign.
EPS = Fraction(1, 1 << 8)


def _det_frac(M):
    n = len(M)
    total = Fraction(0)
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        prod = Fraction(-1 if inv & 1 else 1)
        for r in range(n):
            prod *= M[r][p[r]]
        total += prod
    return total


def _solve(A, b):
    """Gaussian elimination with exact Fractions; None if singular."""
    n = len(A)
    M = [list(map(Fraction, A[i])) + [Fraction(b[i])] for i in range(n)]
    for col in range(n):
        piv = next((r for r in range(col, n) if M[r][col] != 0), None)
        if piv is None:
            return None
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fac = M[r][col] / M[col][col]
                M[r] = [x - fac * y for x, y in zip(M[r], M[col])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _perturbed(V, eps=EPS):
    """V[k][r] + eps^(2^(k*n + r)): vertex k of the face (sorted by id)."""
    n = len(V[0])
    return [[Fraction(V[k][r]) + eps ** (1 << (k * n + r)) for r in range(n)]
            for k in range(len(V))]


def _eq1_punctured(V):
    """Eq. (1): [v_0 .. v_n; 1 .. 1] mu = (0, .., 0, 1); punctured iff every
    mu_j lies in (0, 1).  Returns None for a singular system."""
    n = len(V[0])
    A = [[V[k][r] for k in range(n + 1)] for r in range(n)] + [[1] * (n + 1)]
    b = [0] * n + [1]
    mu = _solve(A, b)
    if mu is None:
        return None
    return all(0 < m < 1 for m in mu)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_sos_sign_equals_concrete_eps(n):
    rng = np.random.default_rng(10 + n)
    for trial in range(400):
        vals = (-1, 0, 1) if trial % 2 else (-2, -1, 0, 1, 2)
        M = rng.choice(vals, size=(n, n))
        if trial < 3:
            M = np.zeros((n, n), dtype=np.int64)
        # entry (r, c) carries local key c*n + r
        Mp = [[Fraction(int(M[r][c])) + EPS ** (1 << (c * n + r)) for c in range(n)]
              for r in range(n)]
        want = 1 if _det_frac(Mp) > 0 else -1
        assert _det_frac(Mp) != 0
        assert cp.sos_det_sign(M) == want, M


def test_sos_2x2_textbook_sequence():
    """Hand expansion of det[[a_x+e^1, b_x+e^4], [a_y+e^2, b_y+e^8]]: the
    decisive terms in increasing exponent are det, b_y, -b_x, -a_y, -1."""
    rng = np.random.default_rng(3)
    for _ in range(500):
        ax, ay, bx, by = (int(v) for v in rng.integers(-2, 3, size=4))
        det = ax * by - ay * bx
        for term in (det, by, -bx, -ay, -1):
            if term != 0:
                want = 1 if term > 0 else -1
                break
        assert cp.sos_det_sign([[ax, bx], [ay, by]]) == want


@pytest.mark.parametrize("n", [2, 3])
def test_predicate_generic_equals_eq1(n):
    """Non-degenerate faces: the predicate is the plain test of Eq. (1)."""
    rng = np.random.default_rng(20 + n)
    hits = 0
    for _ in range(600):
        V = rng.integers(-1000, 1001, size=(n + 1, n))
        # skip degenerate draws (a zero minor)
        minors = [_det_frac([[int(V[j][r]) for j in range(n + 1) if j != k] for r in range(n)])
                  for k in range(n + 1)]
        if any(m == 0 for m in minors):
            continue
        want = _eq1_punctured([[int(x) for x in row] for row in V])
        got = cp.face_punctured(V)
        assert got == want
        hits += want
    assert hits > 20   # both outcomes exercised


@pytest.mark.parametrize("n", [2, 3])
def test_predicate_degenerate_equals_perturbed_eq1(n):
    """Degenerate faces: the predicate is Eq. (1) on the perturbed vectors."""
    rng = np.random.default_rng(30 + n)
    hits = 0
    for trial in range(300 if n == 3 else 800):
        V = rng.integers(-1, 2, size=(n + 1, n))
        if trial == 0:
            V[:] = 0
        want = _eq1_punctured(_perturbed([[int(x) for x in row] for row in V]))
        assert want is not None
        assert cp.face_punctured(V) == want, V
        hits += want
    assert hits > 10


def test_all_zero_face_not_punctured():
    for n in (1, 2, 3):
        assert not cp.face_punctured(np.zeros((n + 1, n), dtype=np.int64))


@pytest.mark.parametrize("dims,nt,seed", [((3, 3), 3, 0), ((4, 3), 2, 1), ((2, 3, 2), 2, 2)])
def test_scan_equals_brute_force(dims, nt, seed):
    """Whole-grid scan (C core) equals enumerating every simplex of the
    spacetime mesh in Python and applying the perturbed Eq. (1)."""
    g = cp.Grid(dims, nt)
    n = g.n
    rng = np.random.default_rng(seed)
    G = rng.integers(-1, 2, size=tuple(reversed(g.dims)) + (n,)).astype(np.int64)
    got = set(int(x) for x in cp.scan_faces(G, g))
    Gf = G.reshape(-1, n)
    want = set()
    for gid in range(g.nverts):
        base = g.coords(gid)
        for ch in g.ftypes:
            if not g.face_exists(base, ch):
                continue
            vids = [g.gid(v) for v in g.simplex_vertices(base, ch)]
            V = [[int(Gf[v][r]) for r in range(n)] for v in vids]
            if _eq1_punctured(_perturbed(V)):
                want.add(g.face_id(base, ch))
    assert got == want
    # ids come back sorted, and the per-id test agrees with the scan
    ids = cp.scan_faces(G, g)
    assert list(ids) == sorted(ids)
    probe = np.arange(g.nverts * g.T, dtype=np.int64)
    res = cp.test_faces(G, g, probe)
    assert set(int(i) for i in probe[res == 1]) == want


def test_order_invariance_within_simplex():
    """Only the order of a simplex's own vertices matters: re-indexing the
    grid with any row-major axis order keeps every Kuhn simplex's vertex order
    (its vertices are componentwise ordered), hence every verdict."""
    g = cp.Grid((3, 3), 3)
    rng = np.random.default_rng(7)
    G = rng.integers(-1, 2, size=(3, 3, 3, 2)).astype(np.int64)
    Gf = G.reshape(-1, 2)
    for gid in range(g.nverts):
        base = g.coords(gid)
        for ch in g.ftypes:
            if not g.face_exists(base, ch):
                continue
            verts = g.simplex_vertices(base, ch)
            for perm in itertools.permutations(range(g.d)):
                # another row-major order: axis perm[0] fastest
                key = lambda c: tuple(c[a] for a in reversed(perm))
                assert sorted(verts, key=key) == verts
            V = [[int(Gf[g.gid(v)][r]) for r in range(2)] for v in verts]
            assert cp.face_punctured(V) == _eq1_punctured(_perturbed(V))
