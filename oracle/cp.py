"""CPU oracle for exact critical-point tracking on the simplicial spacetime mesh.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It
shares no code with the CUDA path (the only common module is the seeded
field sampler ``paper_2011_08697_gb300.synth``, which holds no arithmetic of
the method).

Plain, slow, step-by-step statement of the method (paper Sec. 3.3, Sec. 4):

1. quantise     F = rint(f * 2^S) (round half to even), FP64       (Sec. 4.3)
2. gradient     G_a = F[i+1] - F[i-1]; boundary 2(F[1]-F[0]),
                2(F[N-1]-F[N-2]); each time slice on its own        (Sec. 4.3, 4.7)
3. mesh         Kuhn/Freudenthal subdivision of each unit (n+1)-cube
                (Sec. 3.3): a k-simplex is a base vertex plus a chain
                0 < m_1 < ... < m_k of axis bitmasks
4. predicate    SoS point-in-simplex test, C core ``ftk_oracle.c``  (Sec. 4.3, Eq. 1)
5. location     mu_k = D_k / D from Eq. (1) in FP64 (exact D_k)
6. type         Morse index of the barycentrically weighted,
                symmetrised finite-difference Hessian, exact ints  (Sec. 4.1, Sec. 7)
7. linking      union the punctured faces of every spacetime cell
                (Algorithm 1, left column), label = min face id
8. streaming    ordinal faces at t=k and interval faces of slab
                [k-1, k] become known when slice k arrives          (Sec. 3.2)

Readings where the paper is silent (each listed in the design notes):
the SoS exponent order eps^(2^(g*n+r)); quantise-then-difference; the
one-sided boundary rule; the Hessian-based classification; centroid location
for a fully degenerate puncture.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, exact rational arithmetic, brute force or the paper's printed tables.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(HERE, "libftk_oracle.so")
_SRC = os.path.join(HERE, "ftk_oracle.c")
_SRCS = [_SRC, os.path.join(HERE, "iso_oracle.c")]

RANGE_LIMIT = 1 << 28   # |F| must not exceed 2^28, so |G|, |H| <= 2^30 / 2^31


class OracleRangeError(ValueError):
    pass


# ----------------------------------------------------------------------------
# C core loader
# ----------------------------------------------------------------------------
_lib = None


def build_clib(force: bool = False) -> str:
    """Compile ftk_oracle.c and iso_oracle.c into libftk_oracle.so next to
    them (gcc, -O2, with OpenMP when the compiler has it; the scan then runs
    on several threads)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(x) for x in _SRCS):
        tmp = _SO + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *_SRCS, "-o", tmp]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], stdout=subprocess.DEVNULL,
                          stderr=subprocess.DEVNULL).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def clib():
    global _lib
    if _lib is None:
        build_clib()
        lib = ctypes.CDLL(_SO)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        lib.oracle_sos_det_sign.argtypes = [ctypes.c_int, i64p]
        lib.oracle_sos_det_sign.restype = ctypes.c_int
        lib.oracle_face_punctured.argtypes = [ctypes.c_int, i64p]
        lib.oracle_face_punctured.restype = ctypes.c_int
        lib.oracle_scan.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, i32p,
                                    ctypes.c_int64, ctypes.c_int64, i64p, ctypes.c_int64]
        lib.oracle_scan.restype = ctypes.c_int64
        lib.oracle_scan_mt.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, i32p,
                                       ctypes.c_int64, ctypes.c_int64, i64p, ctypes.c_int64, ctypes.c_int]
        lib.oracle_scan_mt.restype = ctypes.c_int64
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_sos_det_sign_expand.argtypes = [ctypes.c_int, i64p]
        lib.oracle_sos_det_sign_expand.restype = ctypes.c_int
        lib.oracle_test_faces.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, i32p,
                                          i64p, ctypes.c_int64, i8p]
        lib.oracle_test_faces.restype = None
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_iso_edges.argtypes = [ctypes.c_int, i64p, f64p, ctypes.c_double, i64p, ctypes.c_int64]
        lib.oracle_iso_edges.restype = ctypes.c_int64
        lib.oracle_iso_link.argtypes = [ctypes.c_int, i64p, f64p, ctypes.c_double, i64p, ctypes.c_int64,
                                        i64p, i64p]
        lib.oracle_iso_link.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


# ----------------------------------------------------------------------------
# 3. Mesh (Sec. 3.3): chains of axis bitmasks
# ----------------------------------------------------------------------------
def chains(d: int, k: int):
    """All chains 0 < m_1 < m_2 < ... < m_k <= full of nonempty nested axis
    subsets of {0..d-1}, as tuples of bitmasks, in lexicographic order.

    A k-simplex of the subdivided unit d-cube with base vertex v has vertices
    v, v + bits(m_1), ..., v + bits(m_k); the type id of a simplex is the
    index of its chain in this list.
    """
    full = (1 << d) - 1
    out = []
    for combo in itertools.product(range(1, full + 1), repeat=k):
        ok = True
        prev = 0
        for m in combo:
            # strictly nested: prev is a proper subset of m
            if (m & prev) != prev or m == prev:
                ok = False
                break
            prev = m
        if ok:
            out.append(tuple(combo))
    out.sort()
    return out


def face_types(n: int):
    return chains(n + 1, n)


def cell_types(n: int):
    return chains(n + 1, n + 1)


def chain_table(n: int) -> np.ndarray:
    return np.asarray(face_types(n), dtype=np.int32).reshape(-1, n)


class Grid:
    """Spacetime grid: spatial dims (x, y[, z]) plus nt; row-major vertex ids
    g = ((t*Nz + z)*Ny + y)*Nx + x."""

    def __init__(self, dims, nt):
        self.n = len(dims)
        self.d = self.n + 1
        self.dims = tuple(int(v) for v in dims) + (int(nt),)
        self.stride = [1]
        for a in range(1, self.d):
            self.stride.append(self.stride[-1] * self.dims[a - 1])
        self.nverts = self.stride[-1] * self.dims[-1]
        self.ftypes = face_types(self.n)
        self.ctypes_ = cell_types(self.n)
        self.T = len(self.ftypes)
        self.ftype_index = {c: i for i, c in enumerate(self.ftypes)}

    def coords(self, g):
        return tuple((g // self.stride[a]) % self.dims[a] for a in range(self.d))

    def gid(self, c):
        return sum(int(c[a]) * self.stride[a] for a in range(self.d))

    def in_bounds(self, c):
        return all(0 <= c[a] < self.dims[a] for a in range(self.d))

    @staticmethod
    def add_bits(c, m):
        return tuple(c[a] + ((m >> a) & 1) for a in range(len(c)))

    def simplex_vertices(self, base, chain):
        """Vertex coordinates of the simplex (base, chain), in chain order."""
        return [tuple(base)] + [self.add_bits(base, m) for m in chain]

    def face_exists(self, base, chain):
        return self.in_bounds(base) and self.in_bounds(self.add_bits(base, chain[-1]))

    def face_id(self, base, chain):
        return self.gid(base) * self.T + self.ftype_index[tuple(chain)]

    def decode_face(self, fid):
        g, tt = divmod(int(fid), self.T)
        return self.coords(g), self.ftypes[tt]

    # -- cofaces / sides (Sec. 3.2 "side_of()", "sides()") ------------------
    def cofaces(self, base, chain):
        """Cells (base, full chain) that contain the face (base, chain)."""
        d = self.d
        full = (1 << d) - 1
        out = []
        steps = [chain[0]] + [chain[i] ^ chain[i - 1] for i in range(1, len(chain))]
        if chain[-1] == full:
            i = next(j for j, s in enumerate(steps) if bin(s).count("1") == 2)
            prev = chain[i - 1] if i > 0 else 0
            for a in range(d):
                if (steps[i] >> a) & 1:
                    mid = prev | (1 << a)
                    cell = tuple(chain[:i]) + (mid,) + tuple(chain[i:])
                    out.append((tuple(base), cell))
        else:
            a = (full ^ chain[-1]).bit_length() - 1
            # insert the missing axis first: base moves back by e_a
            if base[a] >= 1:
                b2 = tuple(base[j] - (1 if j == a else 0) for j in range(d))
                cell = ((1 << a),) + tuple(m | (1 << a) for m in chain)
                out.append((b2, cell))
            # insert it last
            if base[a] + 1 < self.dims[a]:
                out.append((tuple(base), tuple(chain) + (full,)))
        return out

    def cell_sides(self, base, cell):
        """The d+1 faces (base, chain) of a cell, by dropping one vertex."""
        d = self.d
        out = []
        for k in range(d + 1):
            if k == 0:
                nb = self.add_bits(base, cell[0])
                ch = tuple(m ^ cell[0] for m in cell[1:])
                out.append((nb, ch))
            elif k == d:
                out.append((tuple(base), tuple(cell[:-1])))
            else:
                out.append((tuple(base), tuple(cell[:k - 1]) + tuple(cell[k:])))
        return out


# ----------------------------------------------------------------------------
# 1-2. Quantise and gradient
# ----------------------------------------------------------------------------
def quantise(f: np.ndarray, shift: int = 20) -> np.ndarray:
    """F = rint(f * 2^shift), round half to even, computed in FP64."""
    f64 = np.asarray(f, dtype=np.float32).astype(np.float64)
    if not np.all(np.isfinite(f64)):
        raise OracleRangeError("non-finite sample")
    F = np.rint(f64 * float(2.0 ** shift))
    if np.any(np.abs(F) > RANGE_LIMIT):
        raise OracleRangeError("|f * 2^shift| exceeds 2^28")
    return F.astype(np.int64)


def _fd(A: np.ndarray, axis: int) -> np.ndarray:
    """Integer difference along one array axis: A[i+1]-A[i-1] inside,
    2(A[1]-A[0]) and 2(A[N-1]-A[N-2]) at the two ends."""
    N = A.shape[axis]
    if N < 2:
        raise ValueError("every spatial axis needs at least 2 samples")
    out = np.empty_like(A)

    def sl(s):
        return tuple(s if i == axis else slice(None) for i in range(A.ndim))

    if N > 2:
        out[sl(slice(1, N - 1))] = A[sl(slice(2, N))] - A[sl(slice(0, N - 2))]
    out[sl(slice(0, 1))] = 2 * (A[sl(slice(1, 2))] - A[sl(slice(0, 1))])
    out[sl(slice(N - 1, N))] = 2 * (A[sl(slice(N - 1, N))] - A[sl(slice(N - 2, N - 1))])
    return out


def gradient(F: np.ndarray, n: int) -> np.ndarray:
    """G[..., a] for spatial axis a (0 = x = last array axis)."""
    return np.stack([_fd(F, F.ndim - 1 - a) for a in range(n)], axis=-1)


def hessian(G: np.ndarray, n: int) -> np.ndarray:
    """H[..., a, b] = difference of G_a along spatial axis b (same rule)."""
    base = G.ndim - 1  # array axes of the field come first
    H = np.empty(G.shape + (n,), dtype=np.int64)
    for a in range(n):
        for b in range(n):
            H[..., a, b] = _fd(G[..., a], base - 1 - b)
    return H


# ----------------------------------------------------------------------------
# 4. Predicate (C core) and whole-field scan
# ----------------------------------------------------------------------------
def sos_det_sign(M) -> int:
    """SoS sign of det(M) (columns sorted by vertex id); M is n x n, M[r][c]."""
    M = np.asarray(M, dtype=np.int64)
    n = M.shape[0]
    colmajor = np.ascontiguousarray(M.T).reshape(-1)
    return int(clib().oracle_sos_det_sign(n, _p64(colmajor)))


def face_punctured(V) -> bool:
    """V[k][r]: vector of the k-th vertex (sorted by id). SoS puncture test."""
    V = np.ascontiguousarray(np.asarray(V, dtype=np.int64))
    n = V.shape[1]
    return bool(clib().oracle_face_punctured(n, _p64(V.reshape(-1))))


def sos_det_sign_expand(M) -> int:
    """The same sign from the full expansion (every coefficient)."""
    M = np.asarray(M, dtype=np.int64)
    n = M.shape[0]
    colmajor = np.ascontiguousarray(M.T).reshape(-1)
    return int(clib().oracle_sos_det_sign_expand(n, _p64(colmajor)))


def max_threads() -> int:
    """Threads the C scan can use (1 if it was built without OpenMP)."""
    return int(clib().oracle_max_threads())


def scan_faces(G: np.ndarray, grid: Grid, t_lo: int = 0, t_hi: int | None = None,
               threads: int = 1) -> np.ndarray:
    """Ids (ascending) of all punctured faces with base slice in [t_lo, t_hi).
    ``threads`` > 1 splits the base vertices over OpenMP threads (same ids)."""
    t_hi = grid.dims[-1] if t_hi is None else t_hi
    Gf = np.ascontiguousarray(G.reshape(-1, grid.n).astype(np.int64))
    dims = np.asarray(grid.dims, dtype=np.int64)
    tab = chain_table(grid.n)
    lib = clib()
    cap = 1 << 16
    while True:
        out = np.empty(cap, dtype=np.int64)
        chp = tab.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if threads > 1:
            cnt = lib.oracle_scan_mt(grid.n, _p64(dims), _p64(Gf), grid.T, chp, t_lo, t_hi,
                                     _p64(out), cap, int(threads))
            if cnt < 0:
                raise MemoryError("oracle scan: host allocation failed")
        else:
            cnt = lib.oracle_scan(grid.n, _p64(dims), _p64(Gf), grid.T, chp, t_lo, t_hi, _p64(out), cap)
        if cnt <= cap:
            return out[:cnt].copy()
        cap = int(cnt)


def test_faces(G: np.ndarray, grid: Grid, face_ids) -> np.ndarray:
    """Puncture verdict (1/0, -1 if no such face) for a list of face ids."""
    Gf = np.ascontiguousarray(G.reshape(-1, grid.n).astype(np.int64))
    dims = np.asarray(grid.dims, dtype=np.int64)
    tab = chain_table(grid.n)
    ids = np.ascontiguousarray(np.asarray(face_ids, dtype=np.int64))
    res = np.empty(len(ids), dtype=np.int8)
    clib().oracle_test_faces(grid.n, _p64(dims), _p64(Gf), grid.T,
                             tab.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             _p64(ids), len(ids),
                             res.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return res


# ----------------------------------------------------------------------------
# 5-6. Location and classification (exact integers, then FP64)
# ----------------------------------------------------------------------------
def det_exact(M) -> int:
    """Leibniz formula over permutations, Python integers."""
    n = len(M)
    total = 0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        prod = -1 if inv & 1 else 1
        for r in range(n):
            prod *= int(M[r][p[r]])
        total += prod
    return total


def cramer_numerators(V):
    """D_k = (-1)^(n+k) det(V without vertex k) for Eq. (1); V[k][r]."""
    n = len(V[0])
    out = []
    for k in range(n + 1):
        cols = [V[j] for j in range(n + 1) if j != k]
        M = [[int(cols[c][r]) for c in range(n)] for r in range(n)]
        out.append((-1) ** (n + k) * det_exact(M))
    return out


def barycentric(V):
    """mu_k = D_k / D as exact Fractions (centroid when every D_k is 0)."""
    D = cramer_numerators(V)
    tot = sum(D)
    n1 = len(D)
    if tot == 0:
        return [Fraction(1, n1)] * n1, D
    return [Fraction(dk, tot) for dk in D], D


def morse_index(S) -> int:
    """Number of negative eigenvalues of the symmetric integer matrix S, by
    Descartes' rule on det(lambda I + S) (exact for real-rooted
    polynomials); -1 when det S = 0."""
    n = len(S)
    coeffs = [1]
    for k in range(1, n + 1):
        # e_k = sum of the k x k principal minors
        e = 0
        for idx in itertools.combinations(range(n), k):
            e += det_exact([[S[i][j] for j in idx] for i in idx])
        coeffs.append(e)
    if coeffs[-1] == 0:
        return -1
    nz = [c for c in coeffs if c != 0]
    return sum(1 for a, b in zip(nz, nz[1:]) if (a > 0) != (b > 0))


def classify(D, Hs) -> int:
    """Morse index at a puncture: S = sign(D) * sum_k D_k (H_k + H_k^T)."""
    n = len(Hs[0])
    tot = sum(D)
    sgn = 1 if tot > 0 else (-1 if tot < 0 else 0)
    S = [[0] * n for _ in range(n)]
    for dk, H in zip(D, Hs):
        for a in range(n):
            for b in range(n):
                S[a][b] += sgn * dk * (int(H[a][b]) + int(H[b][a]))
    return morse_index(S)


def classify_vec(D, Js) -> int:
    """Type of a zero of a 2D vector field (Sec. 4.1: sources, sinks and
    saddles from the eigenvalues of the Jacobian): S = sign(D) * sum_k D_k J_k
    is a positive multiple of the barycentrically interpolated Jacobian (not
    symmetrised).  Returns the number of its eigenvalues with negative real
    part: 0 = source, 1 = saddle, 2 = sink; -1 when a real part is zero
    (det S = 0, or det S > 0 with tr S = 0: a centre)."""
    tot = sum(D)
    sgn = 1 if tot > 0 else (-1 if tot < 0 else 0)
    S = [[0, 0], [0, 0]]
    for dk, J in zip(D, Js):
        for a in range(2):
            for b in range(2):
                S[a][b] += sgn * dk * int(J[a][b])
    det = S[0][0] * S[1][1] - S[0][1] * S[1][0]
    tr = S[0][0] + S[1][1]
    if det < 0:
        return 1
    if det == 0 or tr == 0:
        return -1
    return 2 if tr < 0 else 0


# ----------------------------------------------------------------------------
# 7. Linking (Algorithm 1, second pass) with a plain union-find
# ----------------------------------------------------------------------------
class UnionFind:
    def __init__(self):
        self.parent = {}

    def add(self, x):
        self.parent.setdefault(x, x)

    def find(self, x):
        root = x
        while self.parent[root] != root:
            root = self.parent[root]
        while self.parent[x] != root:
            self.parent[x], x = root, self.parent[x]
        return root

    def unite(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            if ra < rb:
                self.parent[rb] = ra
            else:
                self.parent[ra] = rb


class PairingError(AssertionError):
    """A spacetime cell had a punctured-face count other than 0 or 2."""


def cell_pairs(grid: Grid, punct_ids, visit=None, cell_filter=None):
    """Pairs of punctured faces that share a spacetime cell (Algorithm 1,
    second loop): the cells containing a face of ``visit`` (default: every
    punctured face) that pass ``cell_filter(base, cell)``, each checked to
    have 0 or 2 punctured sides (Sec. 4.2, pairing).

    Only cells that contain at least one punctured face can contribute, so
    visiting the cofaces of punctured faces visits every such cell.
    """
    S = set(int(x) for x in punct_ids)
    todo = sorted(S) if visit is None else sorted(int(x) for x in visit)
    seen = set()
    pairs = []
    for f in todo:
        base, chain = grid.decode_face(f)
        for cb, cc in grid.cofaces(base, chain):
            key = (cb, cc)
            if key in seen:
                continue
            seen.add(key)
            if cell_filter is not None and not cell_filter(cb, cc):
                continue
            T = [grid.face_id(sb, sc) for sb, sc in grid.cell_sides(cb, cc)]
            hit = [x for x in T if x in S]
            if len(hit) not in (0, 2):
                raise PairingError(f"cell {key} has {len(hit)} punctured sides")
            if len(hit) == 2:
                pairs.append((hit[0], hit[1]))
    return pairs


def labels_from_pairs(punct_ids, pairs):
    """{face_id: label}: components of the faces under the pairs, label =
    smallest face id of the component."""
    uf = UnionFind()
    for f in punct_ids:
        uf.add(int(f))
    for a, b in pairs:
        uf.unite(a, b)
    return {int(f): uf.find(int(f)) for f in punct_ids}


def link(grid: Grid, punct_ids, cell_filter=None):
    """Union the punctured sides of every cell that has one; returns
    {face_id: label} with label = min face id of the component.
    ``cell_filter(base, cell)`` can restrict the cells (streaming prefixes).
    """
    S = sorted(set(int(x) for x in punct_ids))
    return labels_from_pairs(S, cell_pairs(grid, S, cell_filter=cell_filter))


# ----------------------------------------------------------------------------
# Whole pipeline
# ----------------------------------------------------------------------------
def describe_punctures(grid: Grid, G: np.ndarray, H, ids, classifier=None):
    """Location (Eq. 1), ordinal flag and Morse type (Sec. 4.1) of each
    punctured face in ``ids``; G and H are the gradient / Hessian arrays of
    the grid's vertices (H may be None: types are then left at -2).  For a
    vector field, G holds the vectors, H their Jacobians and ``classifier``
    is ``classify_vec``."""
    classifier = classifier or classify
    n = grid.n
    Gflat = G.reshape(-1, n)
    Hflat = H.reshape(-1, n, n) if H is not None else None
    P = len(ids)
    base = np.zeros((P, 4), dtype=np.int32)
    off = np.zeros((P, 4), dtype=np.float64)
    morse = np.full(P, -2, dtype=np.int8)
    ordinal = np.zeros(P, dtype=np.uint8)
    tbit = 1 << n
    for i, fid in enumerate(ids):
        bc, chain = grid.decode_face(fid)
        verts = grid.simplex_vertices(bc, chain)
        gids = [grid.gid(v) for v in verts]
        V = [[int(Gflat[g][r]) for r in range(n)] for g in gids]
        mu, D = barycentric(V)
        for a in range(n):
            base[i, a] = bc[a]
        base[i, 3] = bc[n]
        ms = [0] + list(chain)
        for a in range(grid.d):
            o = sum(float(mu[k]) for k in range(n + 1) if (ms[k] >> a) & 1)
            off[i, a if a < n else 3] = o
        ordinal[i] = 0 if (chain[-1] & tbit) else 1
        if Hflat is not None:
            morse[i] = classifier(D, [Hflat[g] for g in gids])
    return base, off, morse, ordinal


def track(f: np.ndarray, shift: int = 20, t_lo: int = 0, t_hi: int | None = None,
          with_types: bool = True, with_links: bool = True, threads: int = 1):
    """Exact critical-point tracking of a 2D (nt, ny, nx) or 3D
    (nt, nz, ny, nx) float32 field.

    Returns a dict of numpy arrays, ordered by face id:
      face_id (int64), base (int32, [P, 4] = x, y, z, t), off (float64,
      [P, 4] in-cell offsets), morse (int8), ordinal (uint8), label (int64).
    ``t_lo/t_hi`` restrict the base slices of the faces (a bounded sample).
    ``threads`` is passed to the face scan.
    """
    f = np.asarray(f, dtype=np.float32)
    n = f.ndim - 1
    nt = f.shape[0]
    dims = tuple(reversed(f.shape[1:]))
    grid = Grid(dims, nt)
    F = quantise(f, shift)
    G = gradient(F, n)
    ids = scan_faces(G, grid, t_lo, t_hi, threads=threads)
    H = hessian(G, n) if with_types else None
    base, off, morse, ordinal = describe_punctures(grid, G, H, ids)
    P = len(ids)
    label = np.full(P, -1, dtype=np.int64)
    if with_links and P:
        lab = link(grid, ids)
        label = np.asarray([lab[int(x)] for x in ids], dtype=np.int64)
    return dict(face_id=ids, base=base, off=off, morse=morse, ordinal=ordinal,
                label=label, T=grid.T, grid=grid)


def jacobian(V: np.ndarray, n: int) -> np.ndarray:
    """J[..., a, b] = difference of component a along spatial axis b, with
    the gradient's rule (central inside, one-sided and doubled at the ends)."""
    base = V.ndim - 1
    J = np.empty(V.shape + (n,), dtype=np.int64)
    for a in range(n):
        for b in range(n):
            J[..., a, b] = _fd(V[..., a], base - 1 - b)
    return J


def track_vec(v: np.ndarray, shift: int = 20, with_links: bool = True):
    """Exact tracking of the zeros of a 2D vector field v (nt, ny, nx, 2)
    (paper Sec. 4.1: critical points of a vector field, v(x) = 0): each
    component quantised as in ``quantise``; the puncture predicate, location
    and linking as for a scalar field's gradient, applied to the vectors
    themselves; types from the interpolated Jacobian (``classify_vec``).
    Returns the same arrays as ``track``."""
    v = np.asarray(v, dtype=np.float32)
    if v.ndim != 4 or v.shape[-1] != 2:
        raise ValueError("a 2D vector field has shape (nt, ny, nx, 2)")
    nt, ny, nx, _ = v.shape
    grid = Grid((nx, ny), nt)
    V = quantise(v, shift)
    ids = scan_faces(V, grid)
    J = jacobian(V, 2)
    base, off, morse, ordinal = describe_punctures(grid, V, J, ids, classifier=classify_vec)
    P = len(ids)
    label = np.full(P, -1, dtype=np.int64)
    if with_links and P:
        lab = link(grid, ids)
        label = np.asarray([lab[int(x)] for x in ids], dtype=np.int64)
    return dict(face_id=ids, base=base, off=off, morse=morse, ordinal=ordinal,
                label=label, T=grid.T, grid=grid)


# ----------------------------------------------------------------------------
# The same pipeline spread over host processes, one base slice per task
# ----------------------------------------------------------------------------
def _slab_task(args):
    """Faces with base slice t of the whole field, computed from slices t and
    t+1 alone: gradients and Hessians are per slice (Sec. 4.3), and a face
    with base slice t has its vertices in slices t and t+1.  Ids and base t
    are returned in the whole field's numbering."""
    f_slab, shift, dims, t = args
    n = len(dims)
    sub = Grid(dims, f_slab.shape[0])
    F = quantise(f_slab, shift)
    G = gradient(F, n)
    ids = scan_faces(G, sub, 0, 1)
    H = hessian(G, n)
    base, off, morse, ordinal = describe_punctures(sub, G, H, ids)
    base[:, 3] += t
    shift_ids = t * sub.stride[-1] * sub.T
    return ids + shift_ids, base, off, morse, ordinal


def _pair_task(args):
    """Pairs of the cells whose base vertex lies in slice t: their sides are
    faces with base slice t and ordinal faces of slice t+1."""
    dims, nt, t, S = args
    grid = Grid(dims, nt)
    return cell_pairs(grid, S, cell_filter=lambda cb, cc: cb[-1] == t)


def track_parallel(f: np.ndarray, shift: int = 20, workers: int | None = None):
    """``track`` computed by a pool of host processes (spawned, so the pool
    is safe next to a CUDA context): one task per base slice for detection,
    location and types, one task per slice of cells for the pairs, and the
    union-find over all pairs in this process.  Returns the same arrays as
    ``track``."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    f = np.asarray(f, dtype=np.float32)
    n = f.ndim - 1
    nt = f.shape[0]
    dims = tuple(reversed(f.shape[1:]))
    grid = Grid(dims, nt)
    workers = workers or os.cpu_count() or 1
    tasks = [(np.ascontiguousarray(f[t:t + 2]), shift, dims, t) for t in range(nt)]
    # a worker that dies makes the executor raise (a plain Pool would
    # restart it forever)
    with ProcessPoolExecutor(max_workers=min(workers, nt), mp_context=mp.get_context("spawn")) as pool:
        parts = list(pool.map(_slab_task, tasks))
        ids = np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, np.int64)
        base = np.concatenate([p[1] for p in parts])
        off = np.concatenate([p[2] for p in parts])
        morse = np.concatenate([p[3] for p in parts])
        ordinal = np.concatenate([p[4] for p in parts])
        tbit = 1 << n
        per_t = []
        for t in range(nt):
            own = parts[t][0]
            nxt = []
            if t + 1 < nt:
                nb = parts[t + 1][0]
                types = nb % grid.T
                chains_last = np.asarray([c[-1] for c in grid.ftypes])
                nxt = nb[(chains_last[types] & tbit) == 0]
            per_t.append((dims, nt, t, np.concatenate([own, nxt]).tolist()))
        pairs = list(pool.map(_pair_task, per_t))
    label = np.full(len(ids), -1, dtype=np.int64)
    if len(ids):
        lab = labels_from_pairs(ids.tolist(), [pr for ps in pairs for pr in ps])
        label = np.asarray([lab[int(x)] for x in ids], dtype=np.int64)
    return dict(face_id=ids, base=base, off=off, morse=morse, ordinal=ordinal,
                label=label, T=grid.T, grid=grid)


def _track_task(args):
    f, shift = args
    r = track(f, shift=shift)
    return {k: r[k] for k in ("face_id", "base", "off", "morse", "ordinal", "label")}


def track_many(fields, shift: int = 20, workers: int | None = None):
    """``track`` of many independent fields, one task per field on a pool of
    spawned host processes; returns one result dict per field (without the
    grid object)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = workers or os.cpu_count() or 1
    # largest fields first so that they do not end up last on one worker
    order = sorted(range(len(fields)), key=lambda i: -np.asarray(fields[i]).size)
    out = [None] * len(fields)
    with ProcessPoolExecutor(max_workers=max(1, min(workers, len(fields))),
                             mp_context=mp.get_context("spawn")) as pool:
        for i, r in zip(order, pool.map(_track_task, [(np.asarray(fields[i], dtype=np.float32), shift)
                                                       for i in order])):
            out[i] = r
    return out


# ----------------------------------------------------------------------------
# Trajectories as ordered polylines and their slices at a time t (Sec. 4.1:
# a trajectory is a PL curve in spacetime that can be sliced at t = t0)
# ----------------------------------------------------------------------------
def trajectories(grid: Grid, ids, labels):
    """Each trajectory as its punctured faces in path order.

    Two punctured sides of one cell are consecutive points (the PL field is
    linear in the cell, so its zero set there is the segment between them).
    Returns a list, in increasing label order, of (face ids in path order,
    closed): a path starts at its end with the smaller face id; a loop (no
    ends) starts at its smallest face id and continues to its smaller
    neighbour."""
    ids = [int(x) for x in ids]
    nbr = {f: [] for f in ids}
    for a, b in cell_pairs(grid, ids):
        nbr[a].append(b)
        nbr[b].append(a)
    groups = {}
    for f, lab in zip(ids, [int(x) for x in labels]):
        groups.setdefault(lab, []).append(f)
    out = []
    for lab in sorted(groups):
        members = groups[lab]
        ends = [f for f in members if len(nbr[f]) < 2]
        closed = not ends
        start = min(ends) if ends else min(members)
        order = [start]
        prev, cur = None, start
        while True:
            nxt = [g for g in sorted(nbr[cur]) if g != prev]
            if not nxt or nxt[0] == start:
                break
            prev, cur = cur, nxt[0]
            order.append(cur)
        out.append((order, closed))
    return out


def slice_trajectories(trajs, pos, t0):
    """Crossings of the polylines with the time slice t = t0: one point per
    segment (consecutive points a, b, and the closing segment of a loop)
    with t_a <= t0 < t_b or t_b <= t0 < t_a, interpolated linearly in time.
    ``pos[f]`` = (x, y, z, t) of face f.  Returns a list of
    (label, face_a, face_b, (x, y, z)) with face_a < face_b, grouped by
    trajectory in path order."""
    out = []
    for order, closed in trajs:
        lab = min(order)
        n = len(order)
        segs = [(order[j], order[j + 1]) for j in range(n - 1)]
        if closed and n > 1:
            segs.append((order[-1], order[0]))
        for a, b in segs:
            pa, pb = pos[a], pos[b]
            ta, tb = pa[3], pb[3]
            if not ((ta <= t0 < tb) or (tb <= t0 < ta)):
                continue
            s = (t0 - ta) / (tb - ta)
            xyz = tuple(pa[k] + s * (pb[k] - pa[k]) for k in range(3))
            out.append((lab, min(a, b), max(a, b), xyz))
    return out


def filter_trajectories(trajs, pos, morse, min_duration=0.0, min_points=0, drop_loops=False, half_window=0):
    """Post-processing (Sec. 4.2): keep a trajectory iff its time extent
    (max - min of its points' t) >= min_duration, it has >= min_points
    points and (drop_loops) it is not closed; then smooth the types: a
    point's type becomes the common type of the h points before and the h
    after it along the path when those 2h agree and it differs (loops wrap;
    on a path a point needs h points on each side).  ``morse[f]`` = type of
    face f.  Returns [(order, closed, types)]."""
    out = []
    h = half_window
    for order, closed in trajs:
        ts = [pos[f][3] for f in order]
        n = len(order)
        if n < min_points or max(ts) - min(ts) < min_duration or (drop_loops and closed):
            continue
        types = [int(morse[f]) for f in order]
        new = list(types)
        for j in range(n):
            if h <= 0:
                break
            if closed:
                if n <= 2 * h:
                    continue
                win = [types[(j - q) % n] for q in range(1, h + 1)] + [types[(j + q) % n] for q in range(1, h + 1)]
            else:
                if j < h or j + h >= n:
                    continue
                win = types[j - h:j] + types[j + 1:j + h + 1]
            if all(w == win[0] for w in win) and win[0] != types[j]:
                new[j] = win[0]
        out.append((order, closed, new))
    return out


def positions(result):
    """{face id: (x, y, z, t)} = base + in-cell offset of each puncture."""
    b = result["base"].astype(np.float64)
    o = result["off"]
    return {int(f): tuple(b[i, k] + o[i, k] for k in range(4)) for i, f in enumerate(result["face_id"])}


def stream_push_index(grid: Grid, fid: int) -> int:
    """Push (time slice) after which a face becomes known in a stream:
    ordinal faces at slice t with slice t, interval faces of slab [t, t+1]
    with slice t+1 (Sec. 3.2, ordinal/interval elements)."""
    base, chain = grid.decode_face(fid)
    tbit = 1 << grid.n
    return base[-1] + (1 if chain[-1] & tbit else 0)


def stream_labels(grid: Grid, punct_ids, k: int):
    """Provisional labels known after push k: components over the faces known
    so far, linked through the cells of slabs [t, t+1] with t+1 <= k."""
    known = [int(f) for f in punct_ids if stream_push_index(grid, int(f)) <= k]
    return link(grid, known, cell_filter=lambda cb, cc: cb[-1] + 1 <= k)
