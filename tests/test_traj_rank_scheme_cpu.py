"""CPU model of the trajectory ordering by pointer jumping (the kernels
k_traj_cut, k_traj_rank_init, k_traj_rank_step and k_traj_place, step by
step): on random sets of paths and loops, including two-point loops (the
same pair joined by two cells) and isolated points, every trajectory comes
out in the order of a walk from its smaller end, a loop from its smallest
point towards its smaller neighbour (Sec. 4.1: a trajectory is a PL curve,
its points consecutive along it)."""
import random

import pytest

NO_END = 0x7f7f7f7f
def build_graph(rng, P):
    # random disjoint paths and loops over a random permutation of 0..P-1
    ids = list(range(P)); rng.shuffle(ids)
    nbr = [[-1, -1] for _ in range(P)]
    comps = []
    k = 0
    while k < P:
        L = min(P - k, rng.choice([1, 2, 2, 3, 4, 5, 8, 13, 40, 100]))
        pts = ids[k:k + L]; k += L
        loop = L >= 2 and rng.random() < 0.5
        edges = [(pts[j], pts[j + 1]) for j in range(L - 1)]
        if loop:
            edges.append((pts[-1], pts[0]))   # L == 2: the same pair twice
        for a, b in edges:
            for x, y in ((a, b), (b, a)):
                s = nbr[x]
                s[s.index(-1) if -1 in s else None] = y
        comps.append((pts, loop))
    for s in nbr:
        s.sort()   # -1 first
    return nbr, comps

def serial_order(nbr, pts, loop):
    if loop:
        start = min(pts); order = [start]; prev, cur = None, start
        # towards the smaller neighbour
        nxt = min(nbr[start])
        while nxt != start:
            order.append(nxt); prev, cur = cur, nxt
            a, b = nbr[cur]
            c = [x for x in (a, b) if x != prev]
            nxt = c[0] if c else b
            if len(order) > len(pts): break
        return order
    ends = [p for p in pts if nbr[p][0] < 0]
    start = min(ends); order = [start]; prev, cur = -1, start
    while True:
        a, b = nbr[cur]
        nxt = a if (a >= 0 and a != prev) else (b if b != prev else -1)
        if nxt < 0: break
        order.append(nxt); prev, cur = cur, nxt
    return order

def gpu_model(nbr, comps, P):
    root = [0] * P; start = [NO_END] * P; size = [0] * P
    for pts, loop in comps:
        r = min(pts)
        for p in pts: root[p] = r
        size[r] = len(pts)
        for p in pts:
            if nbr[p][0] < 0: start[r] = min(start[r], p)
    # cut
    nb2 = [0] * (2 * P)
    for i in range(P):
        a, b = nbr[i]; o0, o1 = a, b
        if root[i] == i and start[i] == NO_END: o1 = -1
        if b >= 0 and o1 >= 0 and root[b] == b and start[b] == NO_END and nbr[b][1] == i: o1 = -1
        elif a >= 0 and root[a] == a and start[a] == NO_END and nbr[a][1] == i: o0 = -1
        nb2[2 * i], nb2[2 * i + 1] = o0, o1
    S = []
    for q in range(2 * P):
        i, j = q >> 1, nb2[q]
        S.append((j, i, 1, 0) if j >= 0 else (i, -1, 0, 1))
    maxlen = max(size)
    span = 1
    while span < maxlen:
        T = []
        for q in range(2 * P):
            s = S[q]
            if s[3]: T.append(s); continue
            y, py = s[0], s[1]
            dy = 1 if nb2[2 * y] == py else 0
            t = S[2 * y + dy]
            T.append((t[0], py if t[2] == 0 else t[1], s[2] + t[2], t[3]))
        S = T; span *= 2
    orders = {}
    for i in range(P):
        s0, s1 = S[2 * i], S[2 * i + 1]
        assert s0[3] and s1[3], "walk did not end"
        first = min(s0[0], s1[0])
        rank = s0[2] if s0[0] == first else s1[2]
        r = root[i]
        assert s0[2] + s1[2] + 1 == size[r], ("sizes", i)
        orders.setdefault(r, [None] * size[r])[rank] = i
    return orders



@pytest.mark.parametrize("seed", range(6))
def test_ranking_matches_serial_walk(seed):
    rng = random.Random(seed)
    for _ in range(40):
        P = rng.randint(1, 250)
        nbr, comps = build_graph(rng, P)
        got = gpu_model(nbr, comps, P)
        for pts, loop in comps:
            assert got[min(pts)] == serial_order(nbr, pts, loop)
