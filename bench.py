"""Benchmark: exact critical-point tracking throughput on one GB300.

One step = the whole pipeline (quantise, gradient, cull + exact predicate,
compaction, location, classification, linking, labels) over one synthetic
field already resident in HBM.  Workloads (synthetic stand-ins shaped like
the paper's data):

  spiral2d (default): spiral woven, 1024 x 1024 grid over [-4,4]^2, 64 steps
                      in t in [0,1], + i.i.d. N(0, 1e-3^2), seed = rank
  blobs3d           : 128^3 grid x 16 steps, 32 moving Gaussian blobs

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
}
# bounded CPU-oracle sample per workload: (spatial dims, slices)
ORACLE_SAMPLE = {
    "spiral2d": ((1024, 1024), 2),
    "blobs3d": ((48, 48, 48), 2),
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


def sample_field(wl: str, seed: int):
    """The bounded oracle sample: the same generator law on a smaller grid /
    fewer slices (spiral: the first slices of the full field)."""
    from paper_2011_08697_gb300 import synth
    dims, s = ORACLE_SAMPLE[wl]
    if wl == "spiral2d":
        return synth.spiral_woven(dims[0], WORKLOADS[wl]["nt"], sigma=1e-3, seed=seed,
                                  ny=dims[1], k_stop=s)
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


def profiled_traffic(wl: str):
    """DRAM bytes per detect launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    import hashlib
    src = os.path.join(ROOT, "paper_2011_08697_gb300", "csrc", "ftk_kernels.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"detect_{wl}_traffic.txt")
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


def run_oracle_sample(wl: str, seed: int = 0):
    from oracle import cp
    f = sample_field(wl, seed)
    dims, s = ORACLE_SAMPLE[wl]
    t0 = time.perf_counter()
    r = cp.track(f)
    dt = time.perf_counter() - t0
    return face_count(dims, s), dt, r


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = args.workload
    dims, s = ORACLE_SAMPLE[wl]
    for _ in range(args.warmup):
        run_oracle_sample(wl)
    times = []
    faces = 0
    for _ in range(args.steps):
        faces, dt, _ = run_oracle_sample(wl)
        times.append(dt)
    tot = sum(times)
    value = faces * args.steps / tot
    sample = f"{wl}: {'x'.join(map(str, dims))} grid x {s} slices ({faces} faces) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "simplices/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl]["name"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "simplices/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "simplices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gpu_arm(args):
    import torch
    from paper_2011_08697_gb300 import build as _b, ftk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _b.build()
    lib = ftk.lib()
    wl = args.workload
    W = WORKLOADS[wl]
    f_np = make_field(wl, seed=rank)
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
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                plan.execute(x, stream)
                ends[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    P_check = plan.count()
    assert P_check == P, "puncture count changed between steps"
    my_ms = sum(step_ms)
    tot_ms = my_ms
    if dist is not None:
        t = torch.tensor([my_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = faces * world * args.steps / (tot_ms / 1e3)

    # ---- roofline of the dominant kernel (detect), live CUDA events ---------
    det = []
    stages = []
    with torch.cuda.stream(stream):
        for k in range(max(3, min(args.steps, 20))):
            flush.zero_()
            timed_plan.execute(x, stream)
            timed_plan.count()
            st = timed_plan.stage_times()
            det.append(st[0])
            stages.append(st)
    det_ms = statistics.mean(det)
    alg_bytes = 4.0 * nverts
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (det_ms / 1e3) / 1e9

    # ---- end to end through the C ABI with pinned host buffers -------------
    host = torch.from_numpy(f_np).pin_memory()
    e2e_plan = ftk.Plan(f_np.shape)
    with torch.cuda.stream(stream):
        e2e_plan.execute(host, stream)
        e2e_plan.download()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            e2e_plan.execute(host, stream)
            r = e2e_plan.download()
        e2e_s = time.perf_counter() - t0
    e2e_val = faces * args.steps / e2e_s
    if dist is not None:
        t = torch.tensor([e2e_s], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_val = faces * world * args.steps / float(t.item())

    # ---- bit-exact self-check on the oracle's bounded sample + CPU baseline --
    cpu = None
    exact = None
    if rank == 0 and world == 1 and wl == "spiral2d":
        fs, dt, ref = run_oracle_sample(wl, seed=0)
        sel = (res["base"][:, 3] == 0) | ((res["base"][:, 3] == 1) & (res["ordinal"] == 1))
        exact = bool(np.array_equal(res["face_id"][sel], ref["face_id"])
                     and np.array_equal(res["morse_index"][sel], ref["morse"]))
        dims, s = ORACLE_SAMPLE[wl]
        cpu = {"value": fs / dt, "unit": "simplices/s", "cores": 1, "kind": "oracle",
               "sample": f"{'x'.join(map(str, dims))} grid x {s} slices ({fs} faces), first slices of the workload"}
    elif rank == 0 and world == 1:
        fs, dt, _ = run_oracle_sample(wl, seed=0)
        dims, s = ORACLE_SAMPLE[wl]
        cpu = {"value": fs / dt, "unit": "simplices/s", "cores": 1, "kind": "oracle",
               "sample": f"{'x'.join(map(str, dims))} grid x {s} slices ({fs} faces), same generator law"}

    if rank == 0:
        sm = sorted(step_ms)
        p99 = sm[min(len(sm) - 1, int(round(0.99 * (len(sm) - 1))))]
        line = {
            "metric": METRIC, "value": value, "unit": "simplices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": W["name"], "grid": list(W["dims"]), "nt": W["nt"],
                       "faces_per_step": faces, "vertices_per_step": nverts,
                       "l2": "256 MB buffer written between steps (L2 flushed); steps timed individually",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "timesteps_per_s": W["nt"] * world * args.steps / (tot_ms / 1e3),
            "p50_step_ms": statistics.median(step_ms), "p99_step_ms": p99,
            "punctures": int(P), "trajectories": int(len(np.unique(res["label"]))),
            "bit_exact_sample": exact,
            "stages_ms": {k: statistics.mean(s[i] for s in stages)
                          for i, k in enumerate(["detect", "scan", "finalize", "link", "label"])},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(wl),
                         "kernel": "k_detect", "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": det_ms},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "simplices/s",
                    "h2d_bytes_per_step": int(nverts * 4), "d2h_bytes_per_step": int(P * 56 + 24)},
            "gpu_launches": 5 * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    plan.close()
    timed_plan.close()
    e2e_plan.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="spiral2d")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
