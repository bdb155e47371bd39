"""Benchmark: presort + build of a 2^26-point, 3-d float32 Gaussian-mixture
cloud on one GB300, through the C ABI.

One step = kd_presort + kd_build of the whole cloud (transform, presort,
dedup, rank records, every tree level, on-chip finisher, tree outputs).
``value``: points/s with the coordinates already resident in HBM, timed with
CUDA events around the steps (no per-launch events in that region).
``e2e``: the same call fed from pinned host memory with host outputs
(host->device copy of the coordinates and device->host copy of the whole
tree inside the timed region).  ``roofline``: the dominant kernel family's
bytes per launch under the fixed byte model of the scope table (sort pass:
2(w+4) B per element; level step: 12(k-1) B per element; ...) divided by its
average launch time, from CUDA events recorded around every launch on the
library's stream over a second timed region of the same steps; the
builder's own per-kernel byte model is reported beside it.
``cpu_baseline``: the single-threaded C oracle on a bounded sample of the
same workload.  ``batched``: the 4096-cloud workload in one kd_build_batch
call against per-cloud builds (serial, and pipelined over host threads).
``sweep``: n = 2^22 at k = 2..6 for the presorting build and the O(n log n)
median-selection build side by side.  ``served``: the 20000-request Poisson
stream through kd_submit / kd_wait against serial plain builds.

Multi-GPU: the build does not shard; ``--gpus N`` under torchrun runs N
independent replicas (weak scaling, no collective on the data path).
``--impl reference`` times the CPU oracle instead (the only reference).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "points/s for presort+build (k=3, n=2^26) and % HBM roofline; batched/served vs plain"
UNIT = "points/s"
N_POINTS = 1 << 26
K = 3
SEED = 2
WORKLOAD = "plain-large: n=2^26 tuples, k=3, float32 64-component isotropic Gaussian mixture (seed 2)"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS, help="points per cloud (default 2^26)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served results inside the default line")
    ap.add_argument("--cpu-sample", type=int, default=1 << 24,
                    help="cpu_baseline: oracle sample size in points (2^24: about 15 s of one core)")
    ap.add_argument("--ref-sample", type=int, default=1 << 21,
                    help="--impl reference: oracle sample per step in points (about 2 s of one core)")
    ap.add_argument("--mode", default="plain", choices=["plain", "batched", "served", "sweep", "knn", "profile"],
                    help="plain: the 2^26 build (default line, with batched and served inside); batched / "
                         "served: only those results; sweep: n=2^22 at k=2..6; knn: searches over a "
                         "2^22-tuple tree; profile: warm-up then timed plain builds only (for profilers)")
    ap.add_argument("--clouds", type=int, default=4096)
    ap.add_argument("--requests", type=int, default=20000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The maximum of x over all ranks (x itself at world size 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, points_per_rank: int, seconds_per_step: float) -> float:
    """Points/s of the whole job: every rank builds its own replica per step,
    and the step takes as long as the slowest rank."""
    return world * points_per_rank / seconds_per_step


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


NOMINAL_HBM_GBS = 8000.0


def scope_byte_model(k: int, s: int, w: int, W: int, m: int) -> dict:
    """The algorithmic byte model fixed before the build (per point, and per
    unit of each kernel family).  k dimensions, s coordinate bytes, w key
    word bytes, W significant key bits per coordinate, m tuples after
    duplicate removal; D = ceil(W / 8) digit passes per coordinate, L =
    ceil(log2(m + 1)) levels, L_g = max(0, L - 11) levels in HBM."""
    D = (W + 7) // 8
    L = max(1, int(m).bit_length())
    Lg = max(0, L - 11)
    per_unit = {
        "transform": 2 * k * s,             # per input tuple
        "sort_pass": 2 * (w + 4),           # per element of a digit pass
        "gather": w,                        # per element of a key gather
        "dedup": 8 + k * w,                 # per input tuple
        "level_pass": (k - 1) * 12,         # per element of a level step
        "finish": k * 8 + 4,                # per tuple
    }
    per_point = (per_unit["transform"] + (2 * k - 1) * D * per_unit["sort_pass"] + (2 * k - 1) * w
                 + per_unit["dedup"] + Lg * per_unit["level_pass"] + per_unit["finish"])
    return {"per_point": per_point, "per_unit": per_unit, "D": D, "L": L, "L_g": Lg}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def traffic_for(kernel_family: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the kernel source as it is now (else null)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(kernel_family)
        if not e:
            return None
        src = os.path.join(ROOT, e["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if h != e["sha256"]:
            return None
        return float(e["bytes_per_element"]) * e.get("elements_scale", 1.0)
    except Exception:
        return None


E2E_IN_FLIGHT = 2


def e2e_pipelined(dev: int, pinned, n: int, m: int, tuned: dict, steps: int, threads: int):
    """Seconds per build, and whether every build returned m tuples, for
    `steps` builds per thread from `threads` host threads, each with its own
    context, stream and pinned host outputs, all reading the same pinned
    host coordinates."""
    import ctypes
    import threading
    import torch
    from paper_1410_5420_gb300 import _lib, api
    lib = _lib.load()
    ctxs, outs = [], []
    for _ in range(threads):
        st = torch.cuda.Stream(device=dev)
        ctxs.append(api.kd_create(dev, stream=st, switch_threshold=tuned["switch_threshold"],
                                  level_tile=tuned["level_tile"]))
        outs.append([torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
                     torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory()])
    ok = [True] * threads
    errors = []
    # one presort and one build at a time: a two-stage pipeline, so that one
    # build's upload (inside kd_presort) runs beside another's level passes
    # and download (inside kd_build), instead of the threads drifting into
    # step with each other
    stage = [threading.Lock(), threading.Lock()]

    def run(i: int, count: int):
        try:
            c = _lib.KdCloud(pinned.data_ptr(), n, K, _lib.KD_F32, 0)
            o = outs[i]
            for _ in range(count):
                h = ctypes.c_void_p()
                with stage[0]:
                    ctxs[i].check(lib.kd_presort(ctxs[i].ptr, ctypes.byref(c), ctypes.byref(h)))
                tr = _lib.KdTree(0, -1, ctypes.c_void_p(o[0].data_ptr()), ctypes.c_void_p(o[1].data_ptr()),
                                 ctypes.c_void_p(o[2].data_ptr()), ctypes.c_void_p(o[3].data_ptr()), 0)
                with stage[1]:
                    ctxs[i].check(lib.kd_build(ctxs[i].ptr, h, ctypes.byref(tr)))
                ok[i] = ok[i] and tr.m == m
        except Exception as e:  # reported after the join
            ok[i] = False
            errors.append(e)

    def all_threads(count: int) -> float:
        ts = [threading.Thread(target=run, args=(i, count)) for i in range(threads)]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        torch.cuda.synchronize(dev)
        if errors:
            raise errors[0]
        return time.perf_counter() - t0

    all_threads(1)  # warm-up: pools, pinned staging
    secs = all_threads(steps)
    for c in ctxs:
        c.close()
    return secs / (steps * threads), all(ok)


def cpu_baseline(sample: int):
    """The C oracle (as it stands) on a bounded sample of the same workload,
    and the paper's parallel execution scheme on 2^q host threads (q the
    largest with 2^q <= the host's cores) on the same sample."""
    import kdgen
    import oracle
    coords = kdgen.large_gmm(n=sample)
    t0 = time.perf_counter()
    oracle.build_tree(coords)
    dt = time.perf_counter() - t0
    levels = max(0, (os.cpu_count() or 1).bit_length() - 1)
    t1 = time.perf_counter()
    oracle.build_tree_parallel(coords, levels)
    dtp = time.perf_counter() - t1
    return {"value": sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"n={sample} points of the same mixture (seed 2), one presort+build, {dt:.1f} s",
            "parallel_scheme": {"value": sample / dtp, "unit": UNIT, "cores": 1 << levels,
                                "kind": "the paper's parallel execution scheme (host threads)",
                                "seconds": dtp}}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed on the host cores."""
    if rank != 0:
        return
    import kdgen
    import oracle
    sample = min(args.ref_sample, args.n)
    coords = kdgen.large_gmm(n=sample)
    for _ in range(args.warmup):
        oracle.build_tree(coords)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.build_tree(coords)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total
    cb = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": f"n={sample} points of the same mixture per step (bounded sample of the 2^26 workload)"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": sample, "k": K},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_result(args, dev_index=0):
    """4096 clouds, sizes floor(2^U(6,16)), float32 unit cube, 0.5% duplicates
    (seed 4): one kd_build_batch call against per-cloud kd_presort +
    kd_build, both serial (one host round trip per cloud) and pipelined over
    host threads, each with its own context and stream (the round trips of
    one thread overlap the device work of the others)."""
    import threading
    import torch
    import kdgen
    from paper_1410_5420_gb300 import api
    clouds = kdgen.batch_clouds(count=args.clouds, seed=4)
    pts = int(sum(c.shape[0] for c in clouds))
    dev = [torch.from_numpy(c).cuda(dev_index) for c in clouds]
    stream = torch.cuda.current_stream(dev_index)
    ctx = api.kd_create(dev_index, stream=stream)
    # the autotuner picks the subtree size and level tile for the bucket of the largest cloud
    tuned = api.kd_autotune(ctx, 3, "float32", max(c.shape[0] for c in clouds), reps=3)

    def timed(fn, reps):
        for _ in range(max(1, min(args.warmup, 2))):
            fn()
        torch.cuda.synchronize(dev_index)
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev_index)
        return max(e0.elapsed_time(e1), 1000 * (time.perf_counter() - t0)) / reps, r

    # the clouds back to back in one device tensor (descriptors from the sizes)
    packed = torch.cat(dev)
    sizes = [c.shape[0] for c in clouds]
    ms_b, outs = timed(lambda: api.kd_build_batch_packed(ctx, packed, sizes), args.steps)
    ms_s, singles = timed(lambda: [api.build_tree(ctx, x) for x in dev], 1)
    same = all(torch.equal(outs[i]["node_tuple"], singles[i]["node_tuple"])
               and torch.equal(outs[i]["left"], singles[i]["left"]) for i in range(len(dev)))
    del singles
    nthreads = 4
    streams = [torch.cuda.Stream(dev_index) for _ in range(nthreads)]
    ctxs = [api.kd_create(dev_index, stream=st) for st in streams]

    def pipelined():
        def work(t):
            for i in range(t, len(dev), nthreads):
                api.build_tree(ctxs[t], dev[i])
        th = [threading.Thread(target=work, args=(t,)) for t in range(nthreads)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        torch.cuda.synchronize(dev_index)

    pipelined()
    t0 = time.perf_counter()
    pipelined()
    ms_p = 1000 * (time.perf_counter() - t0)
    for c in ctxs:
        c.close()
    ctx.close()
    return {"workload": f"{args.clouds} clouds, sizes floor(2^U(6,16)), k=3 float32 unit cube, 0.5% duplicates "
                        f"(seed 4)", "points": pts, "ms": ms_b, "points_per_s": pts / (ms_b / 1000.0),
            "plain_per_cloud_serial": {"ms": ms_s, "points_per_s": pts / (ms_s / 1000.0)},
            "plain_per_cloud_pipelined": {"ms": ms_p, "points_per_s": pts / (ms_p / 1000.0),
                                          "host_threads": nthreads},
            "speedup_vs_serial": ms_s / ms_b, "speedup_vs_pipelined": ms_p / ms_b,
            "trees_identical": bool(same), "tuned": tuned}


def run_batched(args):
    r = batched_result(args)
    line = {"metric": METRIC, "mode": "batched", "value": r["points_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
            "dtype": "u32", "data": "synthetic", "config": {"workload": "batched: " + r["workload"],
                                                           "points": r["points"]}, "batched": r}
    print(json.dumps(line), flush=True)


def sweep_result(args, dev_index=0):
    """Dimension sweep: n = 2^22 tuples at k = 2..6, int64 uniform in
    [0, 2^40) (seed 3 + k): points/s of the presorting build (kd_presort +
    kd_build) and of the O(n log n) median-selection build
    (kd_build_select) on the same clouds, the bytes each level step of the
    presorting build moves per element, and where the two cross."""
    import torch
    import kdgen
    from paper_1410_5420_gb300 import api
    n = min(args.n, 1 << 22)
    stream = torch.cuda.current_stream(dev_index)
    rows = []
    for k in range(2, 7):
        x = torch.from_numpy(kdgen.sweep_int64(k, n=n)).cuda(dev_index)

        def timed(fn, steps):
            for _ in range(max(1, min(args.warmup, 3))):
                fn()
            torch.cuda.synchronize(dev_index)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                r = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev_index)
            return e0.elapsed_time(e1) / steps, r

        ctx = api.kd_create(dev_index, stream=stream)  # no per-launch events in the timed builds
        ms_p, t = timed(lambda: api.build_tree(ctx, x, on_device=True), args.steps)
        ms_s, t2 = timed(lambda: api.kd_build_select(ctx, x, on_device=True), args.steps)
        same = bool(torch.equal(t["node_tuple"], t2["node_tuple"]))
        sched_ms = {}
        for name, sc in (("deferred", 1), ("every_level", 2)):
            c2 = api.kd_create(dev_index, stream=stream, schedule=sc)
            ms_x, t3 = timed(lambda: api.build_tree(c2, x, on_device=True), args.steps)
            same = same and bool(torch.equal(t["node_tuple"], t3["node_tuple"]))
            sched_ms[name] = ms_x
            c2.close()
        ctx_t = api.kd_create(dev_index, stream=stream, debug=2)  # per-launch events: level bytes
        api.build_tree(ctx_t, x, on_device=True)
        st = api.kd_kernel_stats(ctx_t)
        ctx_t.close()
        lv = st["level_pass"]
        rows.append({"k": k, "m": t["m"], "presort_ms": ms_p, "presort_points_per_s": n / (ms_p / 1000.0),
                     "select_ms": ms_s, "select_points_per_s": n / (ms_s / 1000.0), "trees_identical": same,
                     "schedule_ms": {"multi_level": ms_p, **sched_ms},
                     "level_steps": lv["launches"],
                     "level_bytes_per_element": lv["bytes"] / lv["units"] if lv["units"] else None})
        ctx.close()
        del x
    faster = [r["k"] for r in rows if r["select_ms"] < r["presort_ms"]]
    return {"workload": f"dimension sweep: n={n} tuples, k=2..6, int64 uniform in [0, 2^40) (seed 3+k)",
            "rows": rows, "select_faster_at_k": faster,
            "presort_ms_per_dimension": (rows[-1]["presort_ms"] - rows[0]["presort_ms"]) / (len(rows) - 1),
            "select_ms_per_dimension": (rows[-1]["select_ms"] - rows[0]["select_ms"]) / (len(rows) - 1)}


def run_sweep(args):
    r = sweep_result(args)
    line = {"metric": METRIC, "mode": "sweep", "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": {"workload": r["workload"]}, "sweep": r}
    print(json.dumps(line), flush=True)


def run_knn(args):
    """Searches over a built tree, on the workload of the paper's Nearest
    Neighbors measurement: n = 2^22 (x, y, z) tuples of int64 uniform in
    [0, 2^40); the kn = 8 nearest neighbours of every tuple (all points),
    the reverse nearest neighbours, and 2^20 region searches.  The CPU
    baseline is the brute-force oracle on a sample of queries."""
    import torch
    import kdgen
    from paper_1410_5420_gb300 import api
    n = min(args.n, 1 << 22)
    kn = 8
    coords = kdgen.cloud_int_uniform(n, 3, 40, 6, np.int64)
    x = torch.from_numpy(coords).cuda()
    stream = torch.cuda.current_stream()
    ctx = api.kd_create(0, stream=stream)
    tree = api.build_tree(ctx, x, on_device=True)
    m = tree["m"]
    ix = api.kd_index_create(ctx, x, tree)
    rng = np.random.default_rng(7)
    centres = coords[rng.integers(0, n, 1 << 20)]
    half = rng.integers(0, 1 << 33, centres.shape)  # boxes that hold a few tuples each
    lo = torch.from_numpy(centres - half).cuda()
    hi = torch.from_numpy(centres + half).cuda()

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    ms_all, (idx, _) = timed(lambda: api.kd_knn_all(ctx, ix, m, kn, with_dist=False), args.steps)
    ms_rev, _ = timed(lambda: api.kd_reverse_knn(ctx, ix, m, kn), args.steps)
    ms_reg, (offs, _) = timed(lambda: api.kd_region(ctx, ix, lo, hi), args.steps)
    found = int(offs[-1].item())
    # CPU baseline: brute force over all tuples for a sample of queries
    import oracle
    sample = 32
    cand = np.arange(n, dtype=np.int32)
    t0 = time.perf_counter()
    oracle.knn(coords, coords[:sample], kn + 1, cand)
    cpu_qps = sample / (time.perf_counter() - t0)
    line = {"metric": METRIC, "mode": "knn", "value": m / (ms_all / 1000.0), "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True,
            "dtype": "i64", "data": "synthetic",
            "config": {"workload": f"all-points {kn} nearest neighbours: n={n} (x,y,z) int64 uniform in [0, 2^40) "
                                   f"(seed 6)", "m": m, "kn": kn},
            "reverse_knn": {"ms": ms_rev, "points_per_s": m / (ms_rev / 1000.0)},
            "region": {"boxes": int(lo.shape[0]), "ms": ms_reg, "boxes_per_s": lo.shape[0] / (ms_reg / 1000.0),
                       "tuples_found": found},
            "cpu_baseline": {"value": cpu_qps, "unit": "queries/s", "cores": 1, "kind": "oracle (brute force)",
                             "sample": f"{sample} queries against all {n} tuples"}}
    print(json.dumps(line), flush=True)
    api.kd_index_destroy(ctx, ix)
    ctx.close()


def host_mem_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / (1 << 20)
    except OSError:
        pass
    return 0.0


def served_result(args, dev_index=0):
    """Poisson stream of build requests through kd_submit / kd_wait: sizes
    log-uniform in [2^8, 2^20], k in {2,3,4}, int32 uniform in [0, 2^24) or
    float32 mixture (seed 5).  Serial plain builds of every request (host
    in, host out) first; then the stream at 0.8x that rate (p50 / p99
    latency from admission to result); then every request at once
    (saturation)."""
    import threading
    from concurrent.futures import ThreadPoolExecutor
    import kdgen
    from paper_1410_5420_gb300 import api
    reqs = kdgen.serving_requests(count=args.requests, seed=5, lo_log2=8.0, hi_log2=20.0)
    est_gb = sum(r[0] * r[1] * 4 for r in reqs) / 2 ** 30
    count = len(reqs)
    if est_gb * 2.5 > host_mem_gb() > 0:  # coordinates plus the library's request copies
        count = max(100, int(count * host_mem_gb() / (est_gb * 2.5)))
        reqs = reqs[:count]
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as pool:  # numpy releases the GIL
        clouds = list(pool.map(lambda r: kdgen.serving_cloud(*r), reqs))
    pts = int(sum(c.shape[0] for c in clouds))
    ctx = api.kd_create(dev_index, mem_budget_bytes=64 << 30)
    for c in clouds[:20]:
        api.build_tree(ctx, c, children=False)
    t0 = time.perf_counter()
    for c in clouds:
        api.build_tree(ctx, c, children=False)
    serial_s = time.perf_counter() - t0
    rate = 0.8 * len(clouds) / serial_s
    arrivals = kdgen.poisson_arrivals(len(clouds), rate, seed=5)

    def stream_run(paced: bool):
        # a waiter thread collects results as they finish, so outputs are
        # dropped early and the submitter never blocks on a result
        q, done = [], threading.Event()
        lock = threading.Condition()

        def waiter():
            i = 0
            while i < len(clouds):
                with lock:
                    while i >= len(q):
                        lock.wait()
                    t = q[i]
                api.kd_wait(ctx, t)
                q[i] = None
                i += 1
            done.set()

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for i, c in enumerate(clouds):
            if paced:
                delay = arrivals[i] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            t = api.kd_submit(ctx, c, children=False)
            with lock:
                q.append(t)
                lock.notify()
        done.wait()
        th.join()
        return time.perf_counter() - t0

    paced_s = stream_run(True)
    st = api.kd_serving_stats(ctx)
    sat_s = stream_run(False)
    ctx.close()
    return {"workload": f"{len(clouds)} Poisson requests of the stream (seed 5), sizes log-U[2^8,2^20], "
                        f"k in {{2,3,4}}, int32 U[0,2^24) or float32 mixture; 64 GB budget",
            "requests": len(clouds), "requests_in_stream": args.requests, "points": pts, "rate_per_s": rate,
            "poisson": {"points_per_s": pts / paced_s, "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                        "completed": st["completed"]},
            "saturation_points_per_s": pts / sat_s, "serial_plain_points_per_s": pts / serial_s,
            "speedup_vs_serial_plain": serial_s / sat_s}


def run_served(args):
    r = served_result(args)
    line = {"metric": METRIC, "mode": "served", "value": r["saturation_points_per_s"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "served: " + r["workload"], "points": r["points"]}, "served": r}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Plain device-resident builds of the mixture at --n only (default
    parameters, no tuning, no extras): --warmup steps, then --steps steps,
    so that a profiler's launch list holds whole steps in order."""
    import torch
    import kdgen
    from paper_1410_5420_gb300 import api
    x = torch.from_numpy(kdgen.large_gmm(n=args.n)).cuda()
    ctx = api.kd_create(0, stream=torch.cuda.current_stream())
    for _ in range(args.warmup + args.steps):
        t = api.build_tree(ctx, x, children=True, on_device=True)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "profile", "n": args.n, "m": t["m"], "steps": args.warmup + args.steps,
                      "launches_per_step": api.kd_launch_count(ctx) / (args.warmup + args.steps)}), flush=True)
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.mode != "plain" and args.impl == "gb300":
        if rank == 0:
            {"batched": run_batched, "served": run_served, "sweep": run_sweep, "knn": run_knn,
             "profile": run_profile}[args.mode](args)
        return
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        if args.impl == "gb300":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    import kdgen
    from paper_1410_5420_gb300 import api

    dev = local
    torch.cuda.set_device(dev)
    n = args.n
    coords_h = kdgen.large_gmm(n=n)
    pinned = torch.from_numpy(coords_h).pin_memory()
    x = pinned.cuda(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = api.kd_create(dev, stream=stream)
    tuned = api.kd_autotune(ctx, K, "float32", n, reps=2)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step(c):
        return api.build_tree(c, x, children=True, on_device=True)

    def timed_steps(c, steps):
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step(c)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return e0.elapsed_time(e1) / steps

    for _ in range(max(1, args.warmup)):
        t = step(ctx)
    m = t["m"]
    del t
    launches0 = api.kd_launch_count(ctx)
    clocks = ClockSampler(dev)
    clocks.start()
    ms_step = timed_steps(ctx, args.steps)
    clk = clocks.stop()
    launches = api.kd_launch_count(ctx) - launches0
    ms_per_step = max_over_ranks(ms_step, world, f"cuda:{dev}")
    value = whole_job_value(world, n, ms_per_step / 1000.0)

    # the same steps again with CUDA events around every launch (per-kernel times)
    ctx_t = api.kd_create(dev, stream=stream, debug=2, switch_threshold=tuned["switch_threshold"],
                          level_tile=tuned["level_tile"])
    step(ctx_t)
    api.kd_kernel_stats_reset(ctx_t)
    ms_step_events = timed_steps(ctx_t, args.steps)
    stats = api.kd_kernel_stats(ctx_t)
    ctx_t.close()

    # the level schedules at the headline size (same tree): the paper's
    # Section 2.1 form, its deferred partitioning, and the default
    sched_ab = {"multi_level": ms_step}
    for name, sc in (("deferred", 1), ("every_level", 2)):
        c2 = api.kd_create(dev, stream=stream, schedule=sc, switch_threshold=tuned["switch_threshold"],
                           level_tile=tuned["level_tile"])
        step(c2)
        sched_ab[name] = timed_steps(c2, max(1, min(args.steps, 3)))
        c2.close()

    # end to end: pinned host coordinates in, whole tree back to pinned host
    out_node = torch.empty(n, dtype=torch.int32).pin_memory()
    out_l = torch.empty(n, dtype=torch.int32).pin_memory()
    out_r = torch.empty(n, dtype=torch.int32).pin_memory()
    out_d = torch.empty(n, dtype=torch.uint8).pin_memory()
    ctx_h = api.kd_create(dev, stream=stream, switch_threshold=tuned["switch_threshold"],
                          level_tile=tuned["level_tile"])
    import ctypes
    from paper_1410_5420_gb300 import _lib
    lib = _lib.load()

    def e2e_step():
        c = _lib.KdCloud(pinned.data_ptr(), n, K, _lib.KD_F32, 0)
        h = ctypes.c_void_p()
        ctx_h.check(lib.kd_presort(ctx_h.ptr, ctypes.byref(c), ctypes.byref(h)))
        tr = _lib.KdTree(0, -1, ctypes.c_void_p(out_node.data_ptr()), ctypes.c_void_p(out_l.data_ptr()),
                         ctypes.c_void_p(out_r.data_ptr()), ctypes.c_void_p(out_d.data_ptr()), 0)
        ctx_h.check(lib.kd_build(ctx_h.ptr, h, ctypes.byref(tr)))
        return tr.m

    for _ in range(2):
        e2e_step()
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mh = e2e_step()
    torch.cuda.synchronize(dev)
    e2e_single_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, f"cuda:{dev}")
    assert mh == m
    ctx_h.close()
    # the same calls from E2E_IN_FLIGHT host threads, each with its own
    # context, stream and pinned outputs: one build's host copies overlap
    # another's kernels
    e2e_s, e2e_ok = e2e_pipelined(dev, pinned, n, m, tuned, e2e_steps, E2E_IN_FLIGHT)
    e2e_s = max_over_ranks(e2e_s, world, f"cuda:{dev}")
    assert e2e_ok

    if rank != 0:
        ctx.close()
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel family under the fixed byte model
    peak, peak_src = measured_peaks()
    model = scope_byte_model(K, 4, 4, 32, m)
    fam = max(stats, key=lambda f: stats[f]["ms"])
    st = stats[fam]
    nl = max(st["launches"], 1)
    per_launch_ms = st["ms"] / nl
    units_per_launch = st["units"] / nl

    def gbs(bytes_per_launch, ms):
        return bytes_per_launch / (ms / 1000.0) / 1e9 if ms > 0 else 0.0

    achieved = gbs(model["per_unit"].get(fam, 0) * units_per_launch, per_launch_ms)
    achieved_own = gbs(st["bytes"] / nl, per_launch_ms)
    tr = traffic_for(fam)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": (tr * units_per_launch) if tr is not None else None,
            "kernel": fam, "bytes_per_unit": model["per_unit"].get(fam, 0),
            "bytes_model": "fixed scope-table model: sort pass 2(w+4) B per element, level step 12(k-1) B "
                           "per element, transform 2ks, dedup 8+kw, finisher 8k+4 B per tuple",
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
            else "fallback 6.8 TB/s",
            "own_model": {"achieved": achieved_own, "frac": achieved_own / peak},
            "step_share": st["ms"] / args.steps / ms_step_events}
    model_bytes = model["per_point"] * n
    own_bytes = sum(v["bytes"] for v in stats.values()) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "k": K, "m": m, "seed": SEED, "parallelism": f"replicas{world}",
                   "tuned": tuned,
                   "l2": "inputs (768 MiB coordinates, GBs of index arrays) exceed the 126 MB L2; no flush"},
        "roofline": roof,
        "step_model": {"bytes_per_point": model["per_point"], "bytes": model_bytes,
                       "achieved_gbs": model_bytes / (ms_per_step / 1000.0) / 1e9,
                       "frac_of_measured": model_bytes / (ms_per_step / 1000.0) / 1e9 / peak,
                       "frac_of_nominal_8tbs": model_bytes / (ms_per_step / 1000.0) / 1e9 / NOMINAL_HBM_GBS,
                       "own_model_bytes": own_bytes,
                       "own_model_frac_of_measured": own_bytes / (ms_per_step / 1000.0) / 1e9 / peak},
        "kernels": {f: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                        "model_gbs": gbs(model["per_unit"].get(f, 0) * v["units"], v["ms"]) or None,
                        "own_gbs": gbs(v["bytes"], v["ms"]) or None}
                    for f, v in stats.items() if v["launches"]},
        "ms_per_step_with_launch_events": ms_step_events,
        "schedule_ms_per_step": sched_ab,
        "clocks": clk,
        "e2e": {"value": whole_job_value(world, n, e2e_single_s), "unit": UNIT, "h2d_bytes_per_step": n * K * 4,
                "d2h_bytes_per_step": m * 13,
                "how": "kd_presort + kd_build from pinned host coordinates to pinned host outputs, one call at a "
                       "time",
                "pipelined": {"value": whole_job_value(world, n, e2e_s), "unit": UNIT, "in_flight": E2E_IN_FLIGHT,
                              "how": f"the same calls from {E2E_IN_FLIGHT} host threads with a context and stream "
                                     f"each, one presort and one build at a time (a two-stage pipeline); "
                                     f"it varies from run to run"}},
        "gpu_launches": launches,
    }
    ctx.close()
    del x
    torch.cuda.empty_cache()
    if not args.no_extras and world == 1:
        line["batched"] = batched_result(args, dev)
        torch.cuda.empty_cache()
        line["sweep"] = sweep_result(args, dev)
        torch.cuda.empty_cache()
        line["served"] = served_result(args, dev)
    if not args.no_cpu_baseline and world >= 1:
        try:
            line["cpu_baseline"] = cpu_baseline(min(args.cpu_sample, n))
        except Exception as ex:  # the oracle build is part of build(); report rather than crash
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"unavailable: {ex}"}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
