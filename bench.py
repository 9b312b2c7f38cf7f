"""Benchmark: exact critical-point tracking throughput on one GB300.

One step = the whole pipeline (quantise, gradient, cull + exact predicate,
compaction, location, classification, linking, labels) over one synthetic
field already resident in HBM.  Workloads (synthetic stand-ins shaped like
the paper's data):

  spiral2d (default): spiral woven, 1024 x 1024 grid over [-4,4]^2, 64 steps
                      in t in [0,1], + i.i.d. N(0, 1e-3^2), seed = rank
  blobs3d           : 128^3 grid x 16 steps, 32 moving Gaussian blobs
  batch2d           : 256 independent 2D blob fields, N log-uniform 64..512,
                      8..32 steps each; one graph-captured batch per step,
                      against a loop of the plain per-field path
  serve2d           : 32 in-situ streams (N log-uniform 256..2048) fed one
                      slice at a time by Poisson arrivals (200 slices/s in
                      total); per-slice latency, then saturated throughput
                      against the plain path run slab by slab

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spacetime simplices tested/s"
WORKLOADS = {
    "spiral2d": dict(name="spiral_woven_1024x1024x64_noise1e-3", ndim=2, dims=(1024, 1024), nt=64),
    "blobs3d": dict(name="gaussian_blobs_128x128x128x16_32blobs", ndim=3, dims=(128, 128, 128), nt=16),
    "batch2d": dict(name="batch_256_blob_fields_N64-512_nt8-32", ndim=2, count=256),
    "serve2d": dict(name="serve_32_streams_N256-2048_poisson200", ndim=2, count=32, rate=200.0),
}
# bounded CPU-oracle sample per workload: (spatial dims, slices), timed on
# all host cores (and the single-core sample, where it is smaller)
ORACLE_SAMPLE = {
    "spiral2d": ((1024, 1024), 2),
    "blobs3d": ((128, 128, 128), 2),
    "batch2d": ((128, 128), 8),
    "serve2d": ((512, 512), 2),
}
SINGLE_SAMPLE = {
    "blobs3d": ((64, 64, 64), 2),
}


def face_count(dims, nt):
    """Number of n-simplices of the Kuhn spacetime mesh of the grid."""
    from itertools import product
    n = len(dims)
    d = n + 1
    ext = tuple(dims) + (nt,)
    full = (1 << d) - 1
    total = 0
    for combo in product(range(1, full + 1), repeat=n):
        prev, ok = 0, True
        for m in combo:
            if (m & prev) != prev or m == prev:
                ok = False
                break
            prev = m
        if not ok:
            continue
        cnt = 1
        for a in range(d):
            cnt *= ext[a] - 1 if (combo[-1] >> a) & 1 else ext[a]
        total += cnt
    return total


def make_field(wl: str, seed: int, dims=None, nt=None):
    from paper_2011_08697_gb300 import synth
    W = WORKLOADS[wl]
    dims = dims or W["dims"]
    nt = nt or W["nt"]
    if wl == "spiral2d":
        return synth.spiral_woven(dims[0], nt, sigma=1e-3, seed=seed, ny=dims[1])
    return synth.gaussian_blobs(dims, nt, nblobs=32, seed=seed)


def sample_field(wl: str, seed: int, single: bool = False):
    """The bounded oracle sample: the same generator law on a smaller grid /
    fewer slices (spiral and blobs at full size: the first slices of the full
    field)."""
    from paper_2011_08697_gb300 import synth
    dims, s = (SINGLE_SAMPLE.get(wl, ORACLE_SAMPLE[wl]) if single else ORACLE_SAMPLE[wl])
    if wl == "spiral2d":
        return synth.spiral_woven(dims[0], WORKLOADS[wl]["nt"], sigma=1e-3, seed=seed,
                                  ny=dims[1], k_stop=s)
    if wl in ("batch2d", "serve2d"):
        # one field of the batch / stream law at a bounded size
        n = dims[0]
        bs = synth.blob_set((n, n), 36, seed=70_000 + seed,
                            sigma_range=(4.0 * n / 128.0, 12.0 * n / 128.0), vmax=1.0)
        return np.stack([synth.blob_slice(bs, k) for k in range(s)])
    return make_field(wl, seed, dims=dims, nt=s)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(wl: str, src_file: str | None = None, name: str | None = None):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary profiles/<name>_traffic.txt, if it was taken on the current
    kernel source (else None): the hash covers the kernel file's device code,
    everything before its host-side marker."""
    import hashlib
    if src_file is None:
        src_file = "ftk_detect3.cu" if wl == "blobs3d" else "ftk_detect2.cu"
    if name is None:
        name = f"detect_{wl}"
    src = os.path.join(ROOT, "paper_2011_08697_gb300", "csrc", src_file)
    text = open(src, "rb").read()
    mark = text.find(b"// ---- host side")
    sha = hashlib.sha256(text if mark < 0 else text[:mark]).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def run_oracle_sample(wl: str, seed: int = 0, threads: int = 1, single: bool = False):
    """The oracle on a bounded sample (``single``: the single-core sample);
    ``threads`` OpenMP threads for the face scan."""
    from oracle import cp
    f = sample_field(wl, seed, single)
    dims, s = (SINGLE_SAMPLE.get(wl, ORACLE_SAMPLE[wl]) if single else ORACLE_SAMPLE[wl])
    t0 = time.perf_counter()
    r = cp.track(f, threads=threads)
    dt = time.perf_counter() - t0
    return face_count(dims, s), dt, r


def reference_arm(args):
    """The oracle as it stands, timed on all host cores (OpenMP face scan) on
    a bounded sample of the workload per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = args.workload
    dims, s = ORACLE_SAMPLE[wl]
    ncpu = os.cpu_count() or 1
    for _ in range(args.warmup):
        run_oracle_sample(wl, threads=ncpu)
    times = []
    faces = 0
    for _ in range(args.steps):
        faces, dt, _ = run_oracle_sample(wl, threads=ncpu)
        times.append(dt)
    tot = sum(times)
    value = faces * args.steps / tot
    metric, unit = METRIC, "simplices/s"
    if wl == "serve2d":
        # one bounded sample = one two-slice slab = one pushed timestep
        value, metric, unit = args.steps / tot, "timesteps/s", "timesteps/s"
    sample = f"{wl}: {'x'.join(map(str, dims))} grid x {s} slices ({faces} faces) per step"
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl]["name"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": unit, "cores": ncpu, "kind": "oracle",
                         "sample": sample + f", face scan on {ncpu} OpenMP threads"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _dist_setup():
    """(dist or None, rank, world, local rank); gloo carries only the
    barrier and the max-over-ranks of the timings."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist, rank, world, local


def _max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank: float, world: int, steps: int, tot_ms: float) -> float:
    """Whole-job throughput of a weak-scaling run: every rank processes its
    own units (an independent replica), the job's time is the slowest rank's."""
    return units_per_rank * world * steps / (tot_ms / 1e3)


def shard_seed(workload: str, rank: int) -> int:
    """Seed of rank's replica: ranks process independent synthetic inputs."""
    return {"batch2d": rank * WORKLOADS["batch2d"]["count"],
            "serve2d": rank * WORKLOADS["serve2d"]["count"]}.get(workload, rank)


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))] if xs else None


def _same_result(a, b) -> bool:
    if len(a) != len(b):
        return False
    if not len(a):
        return True
    return bool(np.array_equal(a["face_id"], b["face_id"]) and np.array_equal(a["label"], b["label"])
                and np.array_equal(a["morse_index"], b["morse_index"])
                and float(np.max(np.abs(a["off"] - b["off"]))) <= 1e-6)


def _oracle_check(res, f) -> bool:
    """Whole-field oracle comparison of one small field (bit-exact faces,
    types and labels; offsets within 1e-5 of a cell)."""
    from oracle import cp
    ref = cp.track(f)
    if not np.array_equal(res["face_id"], ref["face_id"]):
        return False
    return bool(np.array_equal(res["morse_index"], ref["morse"]) and np.array_equal(res["label"], ref["label"])
                and (len(ref["face_id"]) == 0 or float(np.max(np.abs(res["off"] - ref["off"]))) <= 1e-5))


def _cpu_baseline_single(wl):
    """The oracle on one core over the bounded single-core sample."""
    fs, dt, _ = run_oracle_sample(wl, seed=0, threads=1, single=True)
    dims, sl = SINGLE_SAMPLE.get(wl, ORACLE_SAMPLE[wl])
    return {"value": fs / dt, "unit": "simplices/s", "cores": 1, "kind": "oracle",
            "sample": f"{'x'.join(map(str, dims))} grid x {sl} slices ({fs} faces), same generator law"}


def _cpu_baseline(wl):
    """The oracle on all host cores (OpenMP face scan) over the bounded
    sample, with the single-core figure beside it."""
    ncpu = os.cpu_count() or 1
    fs, dt, _ = run_oracle_sample(wl, seed=0, threads=ncpu)
    dims, sl = ORACLE_SAMPLE[wl]
    return {"value": fs / dt, "unit": "simplices/s", "cores": ncpu, "kind": "oracle",
            "sample": f"{'x'.join(map(str, dims))} grid x {sl} slices ({fs} faces), same generator law",
            "single_core": _cpu_baseline_single(wl)}


def batch_arm(args):
    """256 independent fields per step: one graph replay of the batch vs a
    loop of the plain per-field path (plan execute + count per field)."""
    import torch
    from paper_2011_08697_gb300 import build as _b, ftk, synth

    dist, rank, world, local = _dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()
    ftk.lib()
    W = WORKLOADS["batch2d"]
    specs = synth.batch_fields(W["count"], seed0=shard_seed("batch2d", rank), materialise=False)
    xs = [synth.blob_slices_torch(bs, 0, nt, dev) for (n, _, nt, _, bs) in specs]
    shapes = [tuple(x.shape) for x in xs]
    faces = sum(face_count((n, n), nt) for (n, _, nt, _, _) in specs)
    nverts = sum(x.numel() for x in xs)
    steps_per_batch = sum(nt for (_, _, nt, _, _) in specs)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    batch = ftk.Batch(shapes, ftk.make_params(flags=ftk.FTK_FLAG_AUTOTUNE))
    plans = [ftk.Plan(sh) for sh in shapes]
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        batch.execute(xs, stream)                 # uncaptured, autotuned
        tune_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            batch.execute(xs, stream)
            batch.counts()
        for _ in range(max(1, args.warmup // 2)):
            for p, x in zip(plans, xs):
                p.execute(x, stream)
                p.count()
    # exactness: batched == plain on every field; the two smallest fields
    # against the oracle
    got_b = batch.download()
    got_p = [p.download() for p in plans]
    same = all(_same_result(a, b) for a, b in zip(got_b, got_p))
    small = sorted(range(len(specs)), key=lambda i: xs[i].numel())[:2]
    oracle_ok = all(_oracle_check(got_b[i], xs[i].cpu().numpy()) for i in small) if rank == 0 else None
    P = int(sum(len(r) for r in got_b))

    def timed(fn, k):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        with torch.cuda.stream(stream):
            for i in range(k):
                flush.zero_()
                st[i].record(stream)
                fn()
                en[i].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in zip(st, en)]

    def run_batch():
        batch.execute(xs, stream)
        batch.counts()

    def run_plain():
        for p, x in zip(plans, xs):
            p.execute(x, stream)
            p.count()

    def run_plain_async():
        # every field queued on the stream first, then one synchronisation
        # (each count after the first finds its run already complete)
        for p, x in zip(plans, xs):
            p.execute(x, stream)
        for p in plans:
            p.count()

    def barrier():
        if dist is not None:
            dist.barrier()

    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        b_ms = timed(run_batch, args.steps)
    barrier()
    plain_steps = max(3, min(args.steps, 10))
    p_ms = timed(run_plain, plain_steps)
    pa_ms = timed(run_plain_async, plain_steps)
    tot_b = _max_over_ranks(dist, sum(b_ms))
    tot_p = _max_over_ranks(dist, sum(p_ms))
    tot_pa = _max_over_ranks(dist, sum(pa_ms))
    value = weak_value(faces, world, args.steps, tot_b)
    plain_value = weak_value(faces, world, plain_steps, tot_p)
    plain_async_value = weak_value(faces, world, plain_steps, tot_pa)

    # e2e: pinned host fields copied in, batch, results copied out
    hosts = [x.cpu().pin_memory() for x in xs]
    dbuf = [torch.empty_like(x) for x in xs]
    with torch.cuda.stream(stream):
        for h, d in zip(hosts, dbuf):
            d.copy_(h, non_blocking=True)
        batch.execute(dbuf, stream)
        batch.download()
        torch.cuda.synchronize()
        e2e_steps = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for h, d in zip(hosts, dbuf):
                d.copy_(h, non_blocking=True)
            batch.execute(dbuf, stream)
            outs = batch.download()
        e2e_s = _max_over_ranks(dist, time.perf_counter() - t0)
    e2e_val = faces * world * e2e_steps / e2e_s
    kernels = batch.kernels()
    peak, peak_kind = measured_peak_hbm()
    graph_ms = statistics.mean(b_ms)
    achieved = 4.0 * nverts / (graph_ms / 1e3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "simplices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_b / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": W["name"], "fields": len(specs), "faces_per_step": faces,
                       "vertices_per_step": nverts, "timesteps_per_step": steps_per_batch,
                       "l2": "256 MB buffer written between steps (L2 flushed); inputs 1.5 GB > L2",
                       "step": "one CUDA-graph replay of all fields + one counter read-back and check",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "timesteps_per_s": steps_per_batch * world * args.steps / (tot_b / 1e3),
            "p50_step_ms": statistics.median(b_ms), "p99_step_ms": _pct(b_ms, 0.99),
            "plain_loop": {"value": plain_value, "unit": "simplices/s", "ms_per_step": tot_p / plain_steps,
                           "steps": plain_steps,
                           "form": "per field: plan execute + count (synchronising), one stream"},
            "plain_async": {"value": plain_async_value, "unit": "simplices/s",
                            "ms_per_step": tot_pa / plain_steps, "steps": plain_steps,
                            "form": "every field's plan executed on one stream, then one synchronisation"},
            "batched_over_plain": value / plain_value,
            "batched_over_plain_async": value / plain_async_value,
            "autotune_s": tune_s, "punctures": P,
            "bit_exact": {"batched_equals_plain": same, "oracle_two_smallest_fields": oracle_ok},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "whole batch graph",
                         "peak_kind": peak_kind, "algorithmic_bytes_per_launch": 4.0 * nverts,
                         "launch_ms": graph_ms},
            "cpu_baseline": _cpu_baseline("batch2d"),
            "e2e": {"value": e2e_val, "unit": "simplices/s", "h2d_bytes_per_step": int(4 * nverts),
                    "d2h_bytes_per_step": int(P * 56)},
            "gpu_launches": int(kernels * args.steps),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()
    if dist is not None:
        dist.destroy_process_group()


def serve_arm(args):
    """In-situ serving: 32 streams, slices arriving as a Poisson process;
    per-slice latency at that load, then saturated throughput against the
    plain path run on the same slabs one at a time."""
    # one hardware work queue per concurrent stream (the default 8 would make
    # unrelated streams wait on each other); read when CUDA initialises
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_2011_08697_gb300 import build as _b, ftk, synth

    dist, rank, world, local = _dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()
    ftk.lib()
    W = WORKLOADS["serve2d"]
    ns = W["count"]
    specs = synth.stream_specs(ns, seed0=shard_seed("serve2d", rank))
    events = synth.poisson_arrivals(ns, W["rate"], args.duration, seed=rank)
    arrivals = [0] * ns
    for _, s_ in events:
        arrivals[s_] += 1
    n_sat = args.sat_pushes
    slices = [synth.blob_slices_torch(bs, 0, arrivals[i] + n_sat, dev) for i, (n, bs) in enumerate(specs)]
    # the simulation hands over one slice per step: views made once, outside
    # the timed loops (the same for the served and the plain legs)
    views = [[sl[k] for k in range(sl.shape[0])] for sl in slices]
    windows = [[sl[k - 1:k + 1] for k in range(1, sl.shape[0])] for sl in slices]
    torch.cuda.synchronize()
    new_faces = [face_count((n, n), 2) - face_count((n, n), 1) for n, _ in specs]

    budget = int(args.serve_budget_gb * (1 << 30))
    server = ftk.Server(budget)
    streams = [ftk.Stream((n, n), server=server, wait_ms=60_000) for n, _ in specs]
    footprint_open = server.used()
    kpos = [0] * ns               # next slice of each stream
    lat_poisson, lat_sat = [], []
    batch_sizes = []

    # continuous batching from one host thread: every call pushes the slices
    # that have arrived (at most one per stream, in arrival order); slices
    # arriving while a call is on the GPU join the next call
    from collections import deque
    pending = [deque() for _ in range(ns)]
    if dist is not None:
        dist.barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ei, done_n = 0, 0
        while done_n < len(events):
            now = time.perf_counter() - t0
            while ei < len(events) and events[ei][0] <= now:
                pending[events[ei][1]].append(events[ei][0])
                ei += 1
            batch = [i for i in range(ns) if pending[i]]
            if not batch:
                time.sleep(max(0.0, min(1e-3, events[ei][0] - now)))
                continue
            ftk.ftk_streams_push([streams[i] for i in batch], [views[i][kpos[i]] for i in batch])
            t_done = time.perf_counter() - t0
            batch_sizes.append(len(batch))
            for i in batch:
                lat_poisson.append(t_done - pending[i].popleft())
                kpos[i] += 1
                done_n += 1
        poisson_wall = time.perf_counter() - t0
        # saturated: every stream always has a slice waiting
        torch.cuda.synchronize()
        t_sat = time.perf_counter()
        for j in range(n_sat):
            ta = time.perf_counter()
            ftk.ftk_streams_push(streams, [views[i][kpos[i]] for i in range(ns)])
            lat_sat.append(time.perf_counter() - ta)
            for i in range(ns):
                kpos[i] += 1
        sat_wall = time.perf_counter() - t_sat
    total_arrivals = len(events)
    lp = [x * 1e3 for x in lat_poisson]
    ls = [x * 1e3 for x in lat_sat]
    sat_faces = sum(new_faces[i] * n_sat for i in range(ns))
    sat_wall = _max_over_ranks(dist, sat_wall)
    served_steps_s = ns * n_sat * world / sat_wall
    served_faces_s = sat_faces * world / sat_wall

    # plain path on the same slabs, one at a time, one host thread
    plans = {}
    for n, _ in specs:
        if n not in plans:
            plans[n] = ftk.Plan((2, n, n))
    pstream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(pstream):
        for i, (n, _) in enumerate(specs):       # warm-up: every shape once
            plans[n].execute(windows[i][0], pstream)
            plans[n].download()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(n_sat):
            for i, (n, _) in enumerate(specs):
                k = arrivals[i] + j
                plans[n].execute(windows[i][k - 1], pstream)
                plans[n].download()
        plain_wall = _max_over_ranks(dist, time.perf_counter() - t0)
    plain_steps_s = ns * n_sat * world / plain_wall

    # e2e: new streams fed from pinned host slices (the copy is inside push),
    # one batched call per round; two untimed rounds open each stream
    n_e2e = min(8, n_sat)
    hosts = [slices[i][arrivals[i]:arrivals[i] + n_e2e + 2].cpu().pin_memory() for i in range(ns)]
    e2e_streams = [ftk.Stream((n, n)) for n, _ in specs]
    for j in range(2):
        ftk.ftk_streams_push(e2e_streams, [hosts[i][j] for i in range(ns)])
    t0 = time.perf_counter()
    for j in range(2, n_e2e + 2):
        ftk.ftk_streams_push(e2e_streams, [hosts[i][j] for i in range(ns)])
    e2e_wall = _max_over_ranks(dist, time.perf_counter() - t0)
    for s_ in e2e_streams:
        s_.close(False)

    # exactness: the four smallest streams' final results equal the plain
    # path on the whole pushed field; one small stream slab vs the oracle
    order = sorted(range(ns), key=lambda i: specs[i][0])
    same = True
    for i in order[:4]:
        fin = streams[i].close()
        whole = ftk.ftk_track_cp2d(slices[i][: arrivals[i] + n_sat].contiguous())
        same = same and _same_result(fin, whole)
    for i in order[4:]:
        streams[i].close(False)
    used_after = server.used()
    server.close()
    oracle_ok = None
    if rank == 0:
        i = order[0]
        f3 = slices[i][:3].cpu().numpy()
        st = ftk.Stream(f3.shape[1:])
        for k in range(3):
            st.push(f3[k])
        oracle_ok = _oracle_check(st.close(), f3)
    launches_per_push = 1 + 8 + 8  # slice copy, the two-slice pipeline, the stream merge
    if rank == 0:
        line = {
            "metric": "timesteps/s", "value": served_steps_s, "unit": "timesteps/s", "n_gpus": world,
            "steps": ns * n_sat, "warmup": 0, "ms_per_step": 1e3 * sat_wall / (ns * n_sat),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": W["name"], "streams": ns, "grid_N": [n for n, _ in specs],
                       "poisson_rate_steps_s": W["rate"], "poisson_duration_s": args.duration,
                       "saturated_pushes_per_stream": n_sat,
                       "timing": "host wall clock per slice (arrival to delta on the host)",
                       "serving": "continuous batching from one host thread: each ftk_streams_push call "
                                  "takes every slice that has arrived (one per stream)",
                       "l2": "slices of 32 streams (~130 MB per round) rotate through L2; no flush",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "poisson": {"arrivals": total_arrivals, "wall_s": poisson_wall,
                        "mean_batch": statistics.mean(batch_sizes) if batch_sizes else None,
                        "throughput_steps_s": total_arrivals / poisson_wall,
                        "p50_step_ms": _pct(lp, 0.5), "p99_step_ms": _pct(lp, 0.99),
                        "max_step_ms": max(lp) if lp else None},
            "saturated": {"steps_s": served_steps_s, "simplices_s": served_faces_s,
                          "p50_step_ms": _pct(ls, 0.5), "p99_step_ms": _pct(ls, 0.99)},
            "plain_loop": {"value": plain_steps_s, "unit": "timesteps/s",
                           "form": "per slab: 2-slice plan execute + download, one host thread"},
            "served_over_plain": served_steps_s / plain_steps_s,
            "admission": {"budget_bytes": budget, "footprint_bytes_at_open": footprint_open,
                          "footprint_bytes_at_end": used_after, "admitted": ns},
            "bit_exact": {"stream_final_equals_plain_whole_field": same, "oracle_3_slices": oracle_ok},
            "cpu_baseline": _cpu_baseline("serve2d"),
            "e2e": {"value": ns * n_e2e * world / e2e_wall, "unit": "timesteps/s",
                    "h2d_bytes_per_step": int(4 * statistics.mean(n * n for n, _ in specs)),
                    "d2h_bytes_per_step": None},
            "gpu_launches": int(launches_per_push * ns * n_sat),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    for p in plans.values():
        p.close()
    if dist is not None:
        dist.destroy_process_group()


def _pinned_records(n: int):
    """A CP_DTYPE numpy array of n records in pinned host memory (and the
    tensor that owns the memory)."""
    import torch
    from paper_2011_08697_gb300 import ftk
    t = torch.empty(max(1, n) * ftk.CP_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    return t.numpy().view(ftk.CP_DTYPE), t


def _full_oracle_check(res, f):
    """Whole-workload parity against the oracle on all host cores: punctured
    set, Morse index, ordinal flag, base vertex and label equal, offsets
    within 1e-5 of a cell.  Returns (report, oracle seconds, faces)."""
    from oracle import cp
    t0 = time.perf_counter()
    ref = cp.track_parallel(f)
    dt = time.perf_counter() - t0
    ok = bool(np.array_equal(res["face_id"], ref["face_id"]))
    err = None
    if ok:
        ok = all(np.array_equal(res[a], ref[b]) for a, b in
                 (("morse_index", "morse"), ("ordinal", "ordinal"), ("base", "base"), ("label", "label")))
        err = float(np.max(np.abs(res["off"] - ref["off"]))) if len(res) else 0.0
        ok = ok and err <= 1e-5
    return {"full_workload": ok, "punctures": int(len(ref["face_id"])), "max_offset_err": err,
            "compared": "face ids, Morse index, ordinal flag, base vertex, label: equal; offsets <= 1e-5 cell"}, dt, ref


def _measure_plain(wl, args, dev, dist, world, rank, local):
    """One plain-path workload: K timed steps (L2 flushed between steps), the
    dominant kernel's live duration, end to end through the C ABI with pinned
    host buffers."""
    import torch
    from paper_2011_08697_gb300 import ftk
    W = WORKLOADS[wl]
    f_np = make_field(wl, seed=shard_seed(wl, rank))
    nverts = f_np.size
    faces = face_count(W["dims"], W["nt"])
    x = torch.from_numpy(f_np).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    plan = ftk.Plan(f_np.shape)
    timed_plan = ftk.Plan(f_np.shape, ftk.make_params(flags=ftk.FTK_FLAG_STAGE_TIMES))

    def barrier():
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            plan.execute(x, stream)
        P = plan.count()   # settles capacity
        res = plan.download()
        for _ in range(max(args.warmup, 1)):
            timed_plan.execute(x, stream)
        timed_plan.count()

    # ---- timed region: K steps, L2 flushed between steps ------------------
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                plan.execute(x, stream)
                ends[k].record(stream)
        torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    assert plan.count() == P, "puncture count changed between steps"
    tot_ms = _max_over_ranks(dist, sum(step_ms))

    # ---- the dominant kernel (detect), live CUDA events on its stream ------
    det, stages = [], []
    with torch.cuda.stream(stream):
        for k in range(max(3, min(args.steps, 20))):
            flush.zero_()
            timed_plan.execute(x, stream)
            timed_plan.count()
            st = timed_plan.stage_times()
            det.append(st[0])
            stages.append(st)
    det_ms = statistics.mean(det)
    desc = plan.describe()
    streaming = desc["detect_variant"] != 0
    detect_kernel = {0: "k_detect", 1: "k_detect2_stream", 2: "k_detect2_stream<exact>",
                     3: "k_detect3_stream", 4: "k_detect3_stream<exact>"}[desc["detect_variant"]]
    stage_names = (["detect", "survive+scan", "emit+locate", "link", "label"] if streaming
                   else ["detect", "scan", "finalize", "link", "label"])
    alg_bytes = 4.0 * nverts
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (det_ms / 1e3) / 1e9
    step_mean = tot_ms / args.steps

    # ---- end to end through the C ABI: pinned host field in, records out ---
    # Two plans on two streams, as a caller streaming host fields would use
    # them: execute returns once its host copy is done, so the copy of step
    # k+1 overlaps the pipeline of step k; every step's records are
    # downloaded before the next step of that plan.  The one-plan sequence
    # (copy, pipeline, download, in turn) is reported beside it.
    host = torch.from_numpy(f_np).pin_memory()
    outs = [_pinned_records(int(P) + 1024) for _ in range(2)]
    e2e_plans = [ftk.Plan(f_np.shape), ftk.Plan(f_np.shape)]
    e2e_streams = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    for q in range(2):
        e2e_plans[q].execute(host, e2e_streams[q])
        e2e_plans[q].download_into(outs[q][0])
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_plans[0].execute(host, e2e_streams[0])
    for k in range(args.steps):
        a = k & 1
        if k + 1 < args.steps:
            e2e_plans[a ^ 1].execute(host, e2e_streams[a ^ 1])
        r = e2e_plans[a].download_into(outs[a][0])
        assert len(r) == P
    e2e_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_plans[0].execute(host, e2e_streams[0])
        r = e2e_plans[0].download_into(outs[0][0])
    seq_s = time.perf_counter() - t0
    assert len(r) == P
    e2e_val = weak_value(faces, world, args.steps, 1e3 * _max_over_ranks(dist, e2e_s))
    plan.close()
    timed_plan.close()
    for pl_ in e2e_plans:
        pl_.close()
    sm = sorted(step_ms)
    return dict(
        W=W, f_np=f_np, res=res, P=int(P), faces=faces, nverts=nverts, desc=desc, clocks=clk.summary(),
        value=weak_value(faces, world, args.steps, tot_ms), tot_ms=tot_ms, step_ms=step_ms,
        p99=sm[min(len(sm) - 1, int(round(0.99 * (len(sm) - 1))))],
        stages={k: statistics.mean(s[i] for s in stages) for i, k in enumerate(stage_names)},
        roofline={"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                  "frac": achieved / peak, "traffic": profiled_traffic(wl),
                  "kernel": detect_kernel, "peak_kind": peak_kind,
                  "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": det_ms,
                  "whole_step_frac": (alg_bytes / (step_mean / 1e3) / 1e9) / peak},
        e2e={"value": e2e_val, "unit": "simplices/s", "ms_per_step": 1e3 * e2e_s / args.steps,
             "h2d_bytes_per_step": int(nverts * 4), "d2h_bytes_per_step": int(P * 56 + 24),
             "form": "plan execute from a pinned host field + download_into a pinned record buffer; two plans "
                     "on two streams, the host copy of step k+1 overlapping step k",
             "sequential_ms_per_step": 1e3 * seq_s / args.steps},
        gpu_launches=int(desc["kernels_per_execute"]) * args.steps,
    )


ISO_LEVEL = 0.25        # isovalue of the isovolume line: level sets around the positive blobs
ISO_SAMPLE_SLICES = 3   # slices of the bit-exact / CPU-baseline sample of the isovolume line


def edge_count(dims, nt):
    """Number of 1-simplices (edges) of the Kuhn spacetime mesh of the grid:
    sum over nonempty axis masks m of prod_a (N_a - m_a)."""
    ext = tuple(dims) + (nt,)
    d = len(ext)
    total = 0
    for m in range(1, 1 << d):
        cnt = 1
        for a in range(d):
            cnt *= ext[a] - ((m >> a) & 1)
        total += cnt
    return total


def _measure_iso(args, dev, world):
    """Isovolume tracking (Sec. 6.1) of the 128^3 x 16 blob field at
    f = ISO_LEVEL: K timed plan executions (L2 flushed between them), the
    dense edge-bit pass against HBM, a bit-exact comparison with the oracle
    on the first ISO_SAMPLE_SLICES slices, and the oracle's time there."""
    import torch
    from paper_2011_08697_gb300 import ftk
    W = WORKLOADS["blobs3d"]
    f_np = make_field("blobs3d", seed=0)
    nverts = f_np.size
    edges = edge_count(W["dims"], W["nt"])
    x = torch.from_numpy(f_np).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    plan = ftk.IsoPlan(f_np.shape)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            plan.execute(x, ISO_LEVEL, stream)
        P = plan.count()
        res = plan.download()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stages = []
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            plan.execute(x, ISO_LEVEL, stream)
            ends[k].record(stream)
            plan.count()
            stages.append(plan.stage_times())
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    tot_ms = sum(step_ms)
    names = ["edge_bits", "emit", "cell_pass", "label"]
    st = {n: statistics.mean(s[i] for s in stages) for i, n in enumerate(names)}
    bits_ms = st["edge_bits"]
    alg_bytes = 4.0 * nverts + nverts / 8.0      # the field once, one bit per vertex out
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (bits_ms / 1e3) / 1e9
    step_mean = tot_ms / args.steps
    # bit-exact against the oracle on the first slices (the whole pipeline
    # run on that sub-field), and the oracle's time there
    from oracle import iso as oiso
    sub = np.ascontiguousarray(f_np[:ISO_SAMPLE_SLICES])
    got = ftk.ftk_track_iso3d(torch.from_numpy(sub).to(dev), ISO_LEVEL)
    t0 = time.perf_counter()
    ref = oiso.track_iso(sub, ISO_LEVEL)
    dt = time.perf_counter() - t0
    ok = bool(np.array_equal(got["edge_id"], ref["edge_id"]) and np.array_equal(got["label"], ref["label"])
              and np.array_equal(got["base"].astype(np.int64), ref["base"])
              and np.array_equal(got["ordinal"].astype(bool), ref["ordinal"]))
    err = float(np.max(np.abs(got["off"].astype(np.float64) - ref["off"]))) if len(ref["edge_id"]) else 0.0
    sub_edges = edge_count(W["dims"], ISO_SAMPLE_SLICES)
    plan.close()
    return {
        "workload": f"isovolume_f={ISO_LEVEL}_" + W["name"], "metric": "spacetime edges tested/s",
        "value": weak_value(edges, world, args.steps, tot_ms), "unit": "edges/s",
        "ms_per_step": step_mean, "edges_per_step": edges, "intersected_edges": int(P),
        "pieces": int(len(np.unique(res["label"]))), "stages_ms": st,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic("blobs3d", "ftk_iso.cu", "iso_bits_blobs3d"),
                     "kernel": "k_iso_bits",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": bits_ms,
                     "whole_step_frac": (alg_bytes / (step_mean / 1e3) / 1e9) / peak},
        "bit_exact_sample": {"ok": ok, "slices": ISO_SAMPLE_SLICES, "intersected_edges": int(len(ref["edge_id"])),
                             "max_offset_err": err,
                             "compared": "edge ids, labels, base vertices, ordinal flags: equal; offsets <= 1e-5"},
        "cpu_baseline": {"value": sub_edges / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": f"the first {ISO_SAMPLE_SLICES} slices of the workload ({sub_edges} edges)",
                         "seconds": dt},
        "gpu_launches": 4 * args.steps,
    }


VEC_WL = dict(name="vortex_street_512x512x32_24vortices_12sources", dims=(512, 512), nt=32, nvort=24, nsrc=12)
VEC_SAMPLE_SLICES = 3   # slices of the bit-exact / CPU-baseline sample of the vector line


def _measure_vec(args, dev, world):
    """Zeros of a 2D vector field (Sec. 4.1; flow-past-cylinder-shaped
    synthetic wake): K timed plan executions (L2 flushed between them), the
    detect pass in vector mode against HBM (8 bytes per vertex), a
    bit-exact comparison with the oracle on the first VEC_SAMPLE_SLICES
    slices, and the oracle's time there."""
    import torch
    from paper_2011_08697_gb300 import ftk, synth
    W = VEC_WL
    nx, ny = W["dims"]
    v_np = synth.vortex_street(nx, ny, W["nt"], nvort=W["nvort"], nsrc=W["nsrc"], seed=0)
    nverts = nx * ny * W["nt"]
    faces = face_count(W["dims"], W["nt"])
    x = torch.from_numpy(v_np).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    plan = ftk.Plan(v_np.shape, vec2d=True)
    timed = ftk.Plan(v_np.shape, ftk.make_params(flags=ftk.FTK_FLAG_STAGE_TIMES), vec2d=True)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            plan.execute(x, stream)
            timed.execute(x, stream)
        P = plan.count()
        timed.count()
        res = plan.download()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            plan.execute(x, stream)
            ends[k].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    tot_ms = sum(step_ms)
    stages = []
    with torch.cuda.stream(stream):
        for k in range(max(3, min(args.steps, 20))):
            flush.zero_()
            timed.execute(x, stream)
            timed.count()
            stages.append(timed.stage_times())
    desc = plan.describe()
    streaming = desc["detect_variant"] != 0
    names = (["detect", "survive+scan", "emit+locate", "link", "label"] if streaming
             else ["detect", "scan", "finalize", "link", "label"])
    st = {n: statistics.mean(s_[i] for s_ in stages) for i, n in enumerate(names)}
    alg_bytes = 8.0 * nverts
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (st["detect"] / 1e3) / 1e9
    step_mean = tot_ms / args.steps
    from oracle import cp
    sub = np.ascontiguousarray(v_np[:VEC_SAMPLE_SLICES])
    got = ftk.ftk_track_vec2d(torch.from_numpy(sub).to(dev))
    t0 = time.perf_counter()
    ref = cp.track_vec(sub)
    dt = time.perf_counter() - t0
    ok = bool(np.array_equal(got["face_id"], ref["face_id"]))
    err = None
    if ok:
        ok = all(np.array_equal(got[a], ref[b]) for a, b in
                 (("morse_index", "morse"), ("ordinal", "ordinal"), ("base", "base"), ("label", "label")))
        err = float(np.max(np.abs(got["off"] - ref["off"]))) if len(got) else 0.0
        ok = ok and err <= 1e-5
    sub_faces = face_count(W["dims"], VEC_SAMPLE_SLICES)
    plan.close()
    timed.close()
    return {
        "workload": W["name"], "metric": METRIC, "value": weak_value(faces, world, args.steps, tot_ms),
        "unit": "simplices/s", "ms_per_step": step_mean, "punctures": int(P),
        "types": {str(k): int(np.sum(res["morse_index"] == k)) for k in np.unique(res["morse_index"])},
        "stages_ms": st, "plan": desc,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic("vortex2d", "ftk_detect2.cu", "detect_vortex2d") if streaming else None,
                     "kernel": "k_detect2_stream<vector>" if streaming else "k_detect<2> (vector mode)",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": st["detect"],
                     "whole_step_frac": (alg_bytes / (step_mean / 1e3) / 1e9) / peak},
        "bit_exact_sample": {"ok": ok, "slices": VEC_SAMPLE_SLICES, "punctures": int(len(ref["face_id"])),
                             "max_offset_err": err,
                             "compared": "face ids, type, ordinal flag, base vertex, label: equal; offsets <= 1e-5"},
        "cpu_baseline": {"value": sub_faces / dt, "unit": "simplices/s", "cores": 1, "kind": "oracle",
                         "sample": f"the first {VEC_SAMPLE_SLICES} slices of the workload ({sub_faces} faces)",
                         "seconds": dt},
        "gpu_launches": int(desc["kernels_per_execute"]) * args.steps,
    }


TRAJ_FILTER = dict(min_duration=2.0, smooth_half_window=2)


def _measure_traj(f_np, ref, args, dev):
    """Ordered trajectories, their slices at a time t and the filtered,
    type-smoothed trajectories (Sec. 4.1, 4.2) of one tracked field, through
    the C ABI: host wall time per call after a plan execute (each call
    includes its download; the first builds the polylines on the GPU).  With
    the oracle's result ``ref``, every polyline, slice crossing and smoothed
    type is compared with the oracle's walk of its own result."""
    import torch
    from paper_2011_08697_gb300 import ftk
    x = torch.from_numpy(f_np).to(dev)
    nt = f_np.shape[0]
    plan = ftk.Plan(f_np.shape)
    plan.execute(x)
    plan.count()
    res = plan.download()
    ts = res["base"][:, 3].astype(np.float64) + res["off"][:, 3]
    rng = np.random.default_rng(7)
    t_cut = 0.5 * (nt - 1)
    while ts.size and np.min(np.abs(ts - t_cut)) <= 1e-4:   # no point within FP32/FP64 ordering reach
        t_cut = float(rng.uniform(0.25 * (nt - 1), 0.75 * (nt - 1)))
    walk, cut, flt = [], [], []
    for k in range(max(args.steps, 3) + 1):
        plan.execute(x)
        plan.count()
        t0 = time.perf_counter()
        off, pts, closed = plan.trajectories()
        t1 = time.perf_counter()
        sl = plan.slice(t_cut)
        t2 = time.perf_counter()
        foff, fpts, fclosed = plan.trajectories(**TRAJ_FILTER)
        t3 = time.perf_counter()
        if k:                                   # the first round is the warm-up
            walk.append(t1 - t0)
            cut.append(t2 - t1)
            flt.append(t3 - t2)
    plan.close()
    P = len(pts)
    out = {"trajectories": int(len(off) - 1), "points": int(P), "closed": int(np.sum(closed)),
           "slice_t": t_cut, "slice_points": int(len(sl)), "filter": TRAJ_FILTER,
           "kept": int(len(foff) - 1), "kept_points": int(len(fpts)),
           "ms": {"walk": 1e3 * statistics.median(walk), "slice": 1e3 * statistics.median(cut),
                  "filter_smooth": 1e3 * statistics.median(flt)},
           "points_per_s": P / statistics.median(walk),
           "form": "wall time of each C-ABI call after an execute, host results included"}
    if ref is not None:
        from oracle import cp
        trajs = cp.trajectories(ref["grid"], ref["face_id"], ref["label"])
        pos = cp.positions(ref)
        morse = dict(zip(ref["face_id"].tolist(), ref["morse"].tolist()))
        ok = len(off) == len(trajs) + 1
        for i, (order, cl) in enumerate(trajs):
            if not ok:
                break
            ok = pts["face_id"][off[i]:off[i + 1]].tolist() == order and bool(closed[i]) == cl
        want = cp.slice_trajectories(trajs, pos, t_cut)
        ok_s = len(sl) == len(want)
        err = 0.0
        for g, w in zip(sl, want):
            ok_s = ok_s and (int(g["label"]), int(g["face_a"]), int(g["face_b"])) == w[:3]
            err = max(err, float(np.max(np.abs(g["pos"] - np.asarray(w[3])))))
        ok_s = ok_s and err <= 1e-5
        wf = cp.filter_trajectories(trajs, pos, morse, min_duration=TRAJ_FILTER["min_duration"],
                                    half_window=TRAJ_FILTER["smooth_half_window"])
        ok_f = len(foff) == len(wf) + 1
        for i, (order, cl, types) in enumerate(wf):
            if not ok_f:
                break
            ok_f = (fpts["face_id"][foff[i]:foff[i + 1]].tolist() == order and bool(fclosed[i]) == cl
                    and fpts["morse_index"][foff[i]:foff[i + 1]].tolist() == types)
        out["bit_exact"] = {"polylines": bool(ok), "slice": bool(ok_s), "slice_max_pos_err": err,
                            "filtered_smoothed": bool(ok_f),
                            "compared": "every polyline (face ids in path order, closed flag), the slice crossings "
                                        "(label, segment ends; positions <= 1e-5) and the filtered trajectories "
                                        "with smoothed types, against the oracle's walk of its own full result"}
    return out


def gpu_arm(args):
    import torch
    from paper_2011_08697_gb300 import build as _b, ftk

    dist, rank, world, local = _dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()
    ftk.lib()
    wl = args.workload
    m = _measure_plain(wl, args, dev, dist, world, rank, local)
    extra = None
    if args.with_2d and wl == "blobs3d":
        extra = _measure_plain("spiral2d", args, dev, dist, world, rank, local)
    iso_line = None
    if args.with_iso and wl == "blobs3d" and world == 1:
        iso_line = _measure_iso(args, dev, world)
    vec_line = None
    if args.with_vec and wl == "blobs3d" and world == 1:
        vec_line = _measure_vec(args, dev, world)

    if rank == 0:
        W = m["W"]
        line = {
            "metric": METRIC, "value": m["value"], "unit": "simplices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["tot_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": W["name"], "grid": list(W["dims"]), "nt": W["nt"],
                       "faces_per_step": m["faces"], "vertices_per_step": m["nverts"],
                       "l2": "256 MB buffer written between steps (L2 flushed); steps timed individually",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "timesteps_per_s": W["nt"] * world * args.steps / (m["tot_ms"] / 1e3),
            "p50_step_ms": statistics.median(m["step_ms"]), "p99_step_ms": m["p99"],
            "punctures": m["P"], "trajectories": int(len(np.unique(m["res"]["label"]))),
            "stages_ms": m["stages"], "plan": m["desc"], "roofline": m["roofline"],
            "e2e": m["e2e"], "gpu_launches": m["gpu_launches"] + (extra["gpu_launches"] if extra else 0)
            + (iso_line["gpu_launches"] if iso_line else 0) + (vec_line["gpu_launches"] if vec_line else 0),
            "clocks": m["clocks"],
        }
        if extra is not None:
            E = extra["W"]
            line["spiral2d"] = {
                "workload": E["name"], "value": extra["value"], "unit": "simplices/s",
                "ms_per_step": extra["tot_ms"] / args.steps, "p99_step_ms": extra["p99"],
                "timesteps_per_s": E["nt"] * world * args.steps / (extra["tot_ms"] / 1e3),
                "punctures": extra["P"], "stages_ms": extra["stages"], "plan": extra["desc"],
                "roofline": extra["roofline"], "e2e": extra["e2e"], "clocks": extra["clocks"],
                "gpu_launches": extra["gpu_launches"],
            }
        if iso_line is not None:
            line["isovolume"] = iso_line
        if vec_line is not None:
            line["vector2d"] = vec_line
        if world == 1:
            # the oracle on the full workload, all host cores: the bit-exact
            # check and the all-core CPU baseline in one run
            rep, dt, ref3 = _full_oracle_check(m["res"], m["f_np"])
            line["bit_exact"] = rep
            ncpu = os.cpu_count() or 1
            single = _cpu_baseline_single(wl)
            line["cpu_baseline"] = {
                "value": m["faces"] / dt, "unit": "simplices/s", "cores": ncpu, "kind": "oracle",
                "sample": f"the full workload ({m['faces']} faces), one process per base slice on {ncpu} cores",
                "seconds": dt, "single_core": single}
            if args.with_traj:
                line["trajectories_ops"] = _measure_traj(m["f_np"], ref3, args, dev)
            if extra is not None:
                rep2, dt2, _ = _full_oracle_check(extra["res"], extra["f_np"])
                line["spiral2d"]["bit_exact"] = rep2
                line["spiral2d"]["cpu_baseline"] = {
                    "value": extra["faces"] / dt2, "unit": "simplices/s", "cores": ncpu, "kind": "oracle",
                    "sample": "the full workload", "seconds": dt2}
                if args.with_traj:
                    # timing only: the oracle's pure-Python walk of 1.3 M points is not bounded
                    line["spiral2d"]["trajectories_ops"] = _measure_traj(extra["f_np"], None, args, dev)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="blobs3d")
    ap.add_argument("--no-2d", dest="with_2d", action="store_false",
                    help="blobs3d: skip the 2D spiral workload reported beside it")
    ap.add_argument("--no-iso", dest="with_iso", action="store_false",
                    help="blobs3d: skip the isovolume line reported beside it")
    ap.add_argument("--no-vec", dest="with_vec", action="store_false",
                    help="blobs3d: skip the 2D vector-field line reported beside it")
    ap.add_argument("--no-traj", dest="with_traj", action="store_false",
                    help="blobs3d: skip the trajectory walk / slice / filter timings")
    ap.add_argument("--duration", type=float, default=60.0, help="serve2d: Poisson phase seconds")
    ap.add_argument("--sat-pushes", type=int, default=24, help="serve2d: saturated pushes per stream")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0, help="serve2d: admission budget")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batch2d":
        batch_arm(args)
    elif args.workload == "serve2d":
        serve_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
