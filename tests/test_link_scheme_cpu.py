"""The per-cube linking scheme of the CUDA path, modelled on the oracle's mesh
and checked against the oracle's face-driven linking (Algorithm 1, second
loop): every cell lies in one unit cube; a cell is visited only through a
punctured side that contains the cube's base vertex; a cell visited with two
punctured sides joins them, any other nonzero count is an error; and the
cells no cube visits are covered by one global count -- each punctured face
lies in one or two cells, so twice the number of joined cells must equal the
sum of those counts.  On consistent puncture sets (exact SoS results of
degenerate fields) the scheme gives the oracle's components; on sets with a
face removed or added it reports the inconsistency, including the case
where the only offending cell has no punctured side through its base
vertex."""
import itertools

import numpy as np
import pytest

from oracle import cp


def per_cube_link(grid, punct):
    """(components as {face: root}, pairs, incidences, local_errors)."""
    S = set(int(x) for x in punct)
    d = grid.d
    full = (1 << d) - 1
    uf = cp.UnionFind()
    for f in S:
        uf.add(f)
    pairs = errors = 0
    for g in range(grid.nverts):
        b = grid.coords(g)
        if not grid.in_bounds(grid.add_bits(b, full)):
            continue                              # a boundary cube holds no cell
        for cell in cp.cell_types(grid.n):
            sides = [grid.face_id(sb, sc) for sb, sc in grid.cell_sides(b, cell)]
            through_b = [f for (sb, _), f in zip(grid.cell_sides(b, cell), sides) if tuple(sb) == tuple(b)]
            if not any(f in S for f in through_b):
                continue                          # not visited
            hit = [f for f in sides if f in S]
            if len(hit) == 2:
                uf.unite(hit[0], hit[1])
                pairs += 1
            elif hit:
                errors += 1
    incid = 0
    for f in S:
        base, chain = grid.decode_face(f)
        incid += len(grid.cofaces(base, chain))
    return {f: uf.find(f) for f in S}, pairs, incid, errors


def _faces(f):
    r = cp.track(f, with_types=False, with_links=False)
    return r["grid"], [int(x) for x in r["face_id"]]


def _same_partition(a, b):
    def groups(m):
        out = {}
        for f, r in m.items():
            out.setdefault(r, set()).add(f)
        return sorted(sorted(v) for v in out.values())
    return groups(a) == groups(b)


FIELDS = [
    ("2d_ternary", lambda rng: rng.integers(-1, 2, size=(4, 7, 6)).astype(np.float32) * 2.0 ** -20),
    ("2d_smooth", lambda rng: rng.normal(size=(4, 8, 9)).astype(np.float32)),
    ("3d_ternary", lambda rng: rng.integers(-1, 2, size=(3, 4, 5, 4)).astype(np.float32) * 2.0 ** -20),
    ("3d_smooth", lambda rng: rng.normal(size=(3, 5, 4, 5)).astype(np.float32)),
]


@pytest.mark.parametrize("name,make", FIELDS, ids=[n for n, _ in FIELDS])
def test_per_cube_scheme_matches_oracle(name, make):
    rng = np.random.default_rng(7)
    f = make(rng)
    grid, ids = _faces(f)
    assert ids, "fixture must have punctures"
    comp, pairs, incid, errors = per_cube_link(grid, ids)
    assert errors == 0
    assert 2 * pairs == incid
    assert _same_partition(comp, cp.link(grid, ids))


@pytest.mark.parametrize("name,make", FIELDS, ids=[n for n, _ in FIELDS])
def test_inconsistent_sets_are_reported(name, make):
    """Every single-face removal (a broken trajectory) is reported by the
    local check or the global count."""
    rng = np.random.default_rng(11)
    f = make(rng)
    grid, ids = _faces(f)
    for drop in ids[: min(len(ids), 12)]:
        rest = [x for x in ids if x != drop]
        _, pairs, incid, errors = per_cube_link(grid, rest)
        assert errors > 0 or 2 * pairs != incid


def test_unvisited_offending_cell_is_caught_by_the_count():
    """A lone punctured face on the grid's upper boundary whose only cell has
    no punctured side through that cell's base vertex (the face is the side
    opposite it): no cube visits the cell, the count still reports it."""
    grid = cp.Grid((3, 3), 3)
    full = (1 << grid.d) - 1
    for g, cell in itertools.product(range(grid.nverts), cp.cell_types(grid.n)):
        b = grid.coords(g)
        if not grid.in_bounds(grid.add_bits(b, full)):
            continue
        sides = grid.cell_sides(b, cell)
        far = [(sb, sc) for sb, sc in sides if tuple(sb) != tuple(b)]
        assert len(far) == 1
        if len(grid.cofaces(*far[0])) != 1:
            continue            # its other cell would be visited and report it
        fid = grid.face_id(*far[0])
        _, pairs, incid, errors = per_cube_link(grid, [fid])
        assert errors == 0 and pairs == 0 and incid == 1   # only the count sees it
        return
    pytest.fail("no face with a single, unvisited cell in the grid")
