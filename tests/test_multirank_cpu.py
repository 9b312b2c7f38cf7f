"""The multi-rank bench path on CPU: world-size-2 gloo process groups on
127.0.0.1.  Ranks run independent replicas (distinct seeded inputs, no
collective on the data path); the job's time is the slowest rank's and the
whole-job throughput adds every rank's units."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w, local = bench._dist_setup()
    local_ms = 10.0 * (rank + 1)                # rank 1 is the slow one
    tot = bench._max_over_ranks(dist, local_ms)
    value = bench.weak_value(1000.0, w, 5, tot)
    seeds = {wl: bench.shard_seed(wl, r) for wl in ("spiral2d", "blobs3d", "batch2d", "serve2d")}
    f = bench.make_field("spiral2d", bench.shard_seed("spiral2d", r), dims=(16, 12), nt=3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, tot, value, seeds, f))


def test_two_rank_aggregation_and_sharding():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda x: x[0])
    for r, w, tot, value, seeds, f in out:
        assert w == 2
        assert tot == 20.0                     # max over ranks
        assert value == pytest.approx(1000.0 * 2 * 5 / 0.020)
    s0, s1 = out[0][4], out[1][4]
    assert all(s0[k] != s1[k] for k in s0)     # independent replicas
    assert s1["batch2d"] - s0["batch2d"] == 256 and s1["serve2d"] - s0["serve2d"] == 32
    assert not np.array_equal(out[0][5], out[1][5])


def test_single_rank_has_no_process_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w, local = bench._dist_setup()
    assert dist is None and (r, w) == (0, 1)
    assert bench._max_over_ranks(None, 3.5) == 3.5
