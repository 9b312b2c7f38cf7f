"""The index arithmetic of the streaming variants' compaction, modelled on
the CPU: surviving cubes arrive in per-segment runs, the runs in any order
(the compactors claim list space with atomics); a global exclusive prefix
of the cubes' puncture counts over the list, segment totals as differences
across each run, an exclusive scan of those in segment (face-id) order,
stored minus the prefix at the run's start -- so that seg_off[seg] +
surv_off[s] is the sorted position of cube s's first puncture.  The model
must place every puncture at its rank in face-id order, for random run
orders, empty segments and empty cubes."""
import numpy as np
import pytest


def positions(seg_of_run, run_cubes, counts):
    """Model of the kernels: runs laid out in list order (seg_of_run[k] is
    the segment of run k, run_cubes[k] its cubes' per-cube counts)."""
    surv_seg, surv_cnt, run_start = [], [], {}
    for seg, cnts in zip(seg_of_run, run_cubes):
        run_start[seg] = (len(surv_cnt), len(cnts))
        surv_seg += [seg] * len(cnts)
        surv_cnt += list(cnts)
    ns = len(surv_cnt)
    gex = np.concatenate([[0], np.cumsum(surv_cnt)])[:ns] if ns else np.zeros(0, np.int64)   # survivor scan
    total = int(sum(surv_cnt))
    nseg = len(counts)
    seg_off = np.zeros(nseg, np.int64)
    run = 0
    for seg in range(nseg):                               # segment scan, face-id order
        a, n = run_start.get(seg, (0, 0))
        first = int(gex[a]) if n else 0
        end = (int(gex[a + n]) if a + n < ns else total) if n else 0
        seg_off[seg] = run - first
        run += end - first if n else 0
    return [int(seg_off[surv_seg[s]] + gex[s]) for s in range(ns)], surv_seg, surv_cnt, run


@pytest.mark.parametrize("seed", range(20))
def test_positions_are_ranks_in_face_order(seed):
    rng = np.random.default_rng(seed)
    nseg = int(rng.integers(1, 40))
    # per segment: its cubes in vertex order, each with 0..6 punctures
    cubes = [list(rng.integers(0, 7, size=int(rng.integers(0, 9)))) for _ in range(nseg)]
    order = [s for s in rng.permutation(nseg) if cubes[s]]    # runs of non-empty segments, any order
    pos, surv_seg, surv_cnt, P = positions(order, [cubes[s] for s in order], cubes)
    assert P == sum(sum(c) for c in cubes)
    # expected: rank of the first puncture of each cube in (segment, cube) order
    want, r = {}, 0
    for seg in range(nseg):
        for k, c in enumerate(cubes[seg]):
            want[(seg, k)] = r
            r += int(c)
    seen = {}
    for s, (seg, p) in enumerate(zip(surv_seg, pos)):
        k = seen.get(seg, 0)
        seen[seg] = k + 1
        assert p == want[(seg, k)]
