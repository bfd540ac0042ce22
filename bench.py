"""Benchmark of the CRK-HACC short-range pair path on GB300: pair interactions/s.

One step = the whole hot path over one box: leaf build (RCB), geometry,
corrections, hydro (acceleration + energy), short-range gravity, the gravity
adjoint (cotangent 2a) and the geometry adjoint (cotangent 1 on every gas
density).  ``value`` = ordered in-range pair interactions processed by all
kernels of a step x steps / device time (inputs resident in HBM), summed over
ranks.  Pair counts are the kernels' own in-range counts from an untimed
counting step.

``--impl reference`` times the FP64 CPU oracle (the only reference this
path has) on a bounded sample of the same workload.

Launch: python bench.py [--gpus N --steps K --warmup W --workload NAME]
(N > 1 through torch.distributed.run: independent replica boxes, one per rank).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# algorithmic FP32 operations per in-range pair (FMA = 2, add/mul = 1; MUFU counted apart),
# counted from the operations of each kernel's pair term (e.g. gravity: d 3, r^2 5, +eps^2 1,
# r^-3 2, Horner P5 10, g 1, m g 1, three FMAs 6)
FLOPS_PER_PAIR = {"geometry": 24, "corrections": 88, "hydro": 160, "gravity": 29, "gravity_adjoint": 68,
                  "geometry_adjoint": 31}
MUFU_PER_PAIR = {"geometry": 2, "corrections": 2, "hydro": 3, "gravity": 1, "gravity_adjoint": 1,
                 "geometry_adjoint": 2}
STAGES = ["leaves", "geometry", "corrections", "hydro", "gravity", "gravity_adjoint", "geometry_adjoint"]
# DRAM bytes (read + write) per launch of a kernel in one launch shape (workload, kernel, variant,
# depth, warps), from one ncu capture of the current build (dram__bytes_read.sum + dram__bytes_write.sum;
# the summaries under profiles/ give the commands).  A shape not captured since its kernel last
# changed has no entry, and the bench line then reports traffic null.  The large box's entries are the
# medium-box captures (307.1 MB in both shapes) scaled by the in-range pairs per launch (8.784e9 / 1.328e9).
TRAFFIC = {("large", "gravity_adjoint", 1, 96, 2): 2.032e9, ("large", "gravity_adjoint", 1, 96, 4): 2.032e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="crk", choices=["crk", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "medium", "clustered", "adjoint", "tiny"])
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--trace-leaves", action="store_true", help="after timing, print leaf-build phase times")
    ap.add_argument("--variants", default="", help="kernel=variant,... (0 lists, 1 tiles, 2 tiles16, 3 tiles8, 4 ring16, 5-7 half-warp, "
                                                     "8 split8)")
    ap.add_argument("--launch", default="", help="kernel=P:D:W,... launch shapes (persistent 0/1, j-tile depth, "
                                                   "warps per block) instead of the autotuner's (profiling runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain measurement")
    ap.add_argument("--no-extras", action="store_true", help="skip the Extras-chain measurement")
    ap.add_argument("--no-advance", action="store_true", help="skip the timestep/integrator measurement")
    ap.add_argument("--no-adjoint-chain", action="store_true",
                    help="skip the corrections/hydro adjoint measurement")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the corrections/hydro adjoint measurement (--steps calls each) and print it")
    ap.add_argument("--advance-only", action="store_true",
                    help="run only the timestep/integrator measurement (--steps steps) and print it")
    ap.add_argument("--no-tune", action="store_true", help="keep the default kernel variants")
    ap.add_argument("--batched-boxes", type=int, default=96)
    return ap.parse_args()


def make_box(name, rank):
    from paper_2310_16122_gb300 import workloads as W

    if name == "large":
        b = W.clustered_box(256, 5000, W.SEEDS["large"] + 7919 * rank, name="large_2x256^3")
    elif name == "medium":  # profiling case: 2x128^3, inputs larger than L2
        b = W.clustered_box(128, 1600, W.SEEDS["large"] + 31 + 7919 * rank, name="medium_2x128^3")
    elif name == "clustered":
        b = W.clustered_box(64, 200, W.SEEDS["clustered"] + 7919 * rank, name="clustered_2x64^3")
    elif name == "adjoint":
        b = W.clustered_box(32, 25, W.SEEDS["adjoint"] + 7919 * rank, name="adjoint_2x32^3")
    else:
        b = W.lattice_box(16, 0.2, W.SEEDS["tiny"] + 7919 * rank, h=1.0, leaf_mode=0, cells=4, name="tiny_2x16^3")
    return b


class Clocks:
    """nvidia-smi sampler during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def aggregate(ms, pairs, dist=None, device="cpu"):
    """Whole-job figures over ranks: the slowest rank's time and the sum of every rank's pairs."""
    if dist is None:
        return float(ms), float(pairs)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0]), float(p[0])


def run_reference(args, rank):
    """The oracle as it stands, on a bounded sample of the same workload, on the host cores."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2310_16122_gb300 import workloads as W
    import numpy as np

    box = make_box(args.workload, 0)
    I = O.from_box(box)
    threads = O.num_threads()
    sample_n = args.cpu_sample or (64 if args.workload == "large" else 256)
    rng = np.random.default_rng(12345)
    for _ in range(args.warmup):
        O.sampled_chain(I, rng.choice(box.n, 8, replace=False), W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
    pairs, t = 0, 0.0
    for _ in range(args.steps):
        s = rng.choice(box.n, sample_n, replace=False)
        t0 = time.perf_counter()
        r = O.sampled_chain(I, s, W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
        t += time.perf_counter() - t0
        pairs += r["pairs"]
    value = pairs / t
    sample = (f"{sample_n} random particles per step of the {box.name} box: geometry on their two-hop gas "
              f"neighbourhood, corrections on the one-hop, hydro and gravity adjoint on the sample, gravity "
              f"on its gravity neighbourhood (FP64 oracle, OpenMP)")
    line = {"impl": "reference", "metric": "pair interactions/s per GB300 (fwd & adjoint)", "value": value,
            "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": box.name, "n_particles": box.n, "box": box.L, "sample": sample_n},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(box, seconds=10.0):
    """Oracle pairs/s on a bounded sample of the workload (host cores).

    The oracle rebuilds its cell lists over the whole box on every call, so
    the sample grows until one call takes about `seconds`; that call is timed.
    """
    from oracle import oracle as O
    from paper_2310_16122_gb300 import workloads as W
    import numpy as np

    I = O.from_box(box)
    rng = np.random.default_rng(2024)
    n_s, spent = 256, 0.0
    while True:
        s = rng.choice(box.n, min(n_s, box.n), replace=False)
        t0 = time.perf_counter()
        r = O.sampled_chain(I, s, W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
        dt = time.perf_counter() - t0
        spent += dt
        if dt >= seconds or n_s >= box.n or spent > 4 * seconds:
            break
        n_s = int(min(box.n, n_s * max(2.0, 1.2 * seconds / max(dt, 1e-3))))
    cores = O.num_threads()
    # the same chain on one host core, on a sixteenth of the sample
    s1 = s[: max(64, s.size // 16)]
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        r1 = O.sampled_chain(I, s1, W.GAMMA, W.AV_ALPHA, W.AV_BETA, W.AV_ETA2)
        dt1 = time.perf_counter() - t0
    finally:
        O.set_threads(cores)
    return r, s, {"value": r["pairs"] / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{s.size} random i-particles of the same box through the oracle's sampled chain (geometry "
                      f"on their two-hop gas neighbourhood, corrections one-hop, hydro, gravity on the gravity "
                      f"neighbourhood, gravity adjoint); {r['pairs']} pairs in {dt:.1f} s",
            "one_core": {"value": r1["pairs"] / dt1, "unit": "pairs/s", "cores": 1,
                         "sample": f"{s1.size} of the same particles; {r1['pairs']} pairs in {dt1:.1f} s"}}


def error_stats(got, ref):
    """E = sqrt(sum|d|^2 / sum|ref|^2) and the per-particle e_i = |d_i| / (|ref_i| + 0.01 rms|ref|)."""
    import numpy as np

    r = np.asarray(ref, np.float64).reshape(len(ref), -1)
    g = np.asarray(got, np.float64).reshape(len(ref), -1)
    d = np.linalg.norm(g - r, axis=1)
    a = np.linalg.norm(r, axis=1)
    e = d / (a + 0.01 * float(np.sqrt(np.mean(a * a))) + 1e-300)
    return {"E": float(np.sqrt(np.sum(d * d) / max(np.sum(a * a), 1e-300))), "median": float(np.median(e)),
            "p99": float(np.percentile(e, 99)), "max": float(e.max()), "n": int(len(e))}


def sample_errors(api, ctx, db, box, ref, sample):
    """Error of every step output against the oracle's sampled chain (the cpu_baseline sample):
    one untimed crk_step with every intermediate returned, on fresh leaves."""
    import torch

    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    io = api.StepIO(ctx, db)
    api.step(ctx, lv, db, io)
    torch.cuda.synchronize()
    gas_s = sample[box.species[sample] == 0]
    T = lambda t: t.cpu().numpy().T if t.dim() == 2 else t.cpu().numpy()
    out = {}
    for k, t in (("acc", io.acc), ("gx", io.gx_grav), ("gm", io.gm_grav)):
        out[k] = error_stats(T(t)[sample], ref[k][sample])
    for k, t in (("dv", io.dv), ("du", io.du), ("V", io.V), ("rho", io.rho), ("A", io.A), ("B", io.B),
                 ("gA", io.gA), ("gB", io.gB)):
        out[k] = error_stats(T(t)[gas_s], ref[k][gas_s])
    lv.free()
    return {"sample": f"{sample.size} particles of the cpu_baseline sample ({gas_s.size} gas)", "outputs": out}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2310_16122_gb300 import api, native
    from paper_2310_16122_gb300.build import build_library

    build_library()
    box = make_box(args.workload, rank)
    ctx = api.Context(local)
    for kv in filter(None, args.variants.split(",")):
        k, v = kv.split("=")
        ctx.set_variant(k, int(v))
    for kv in filter(None, args.launch.split(",")):
        k, v = kv.split("=")
        pm, d, w = (int(t) for t in v.split(":"))
        ctx.set_launch(k, pm, d, w)
    variants = {k: ctx.get_variant(k) for k in native.KERNELS}
    db = api.DeviceBox(box, device=f"cuda:{local}")
    gas = (db.species == 0).float()
    stream = ctx.stream
    if args.adjoint_only:
        # the adjoint row alone (for kernel launch lists of the adjoints); not the headline line
        try:
            f_max = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0))
        except Exception:
            f_max = 2070.0
        peak = torch.cuda.get_device_properties(local).multi_processor_count * 128 * 2 * f_max * 1e6 / 1e12
        if rank == 0:
            print(json.dumps({"workload": box.name, "n": box.n,
                              "adjoint_chain": adjoint_chain(api, ctx, db, stream, peak, reps=args.steps)}))
        return
    if args.advance_only:
        # the timestep row alone (for kernel launch lists of crk_advance); not the headline line
        try:
            f_max = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0))
        except Exception:
            f_max = 2070.0
        peak = torch.cuda.get_device_properties(local).multi_processor_count * 128 * 2 * f_max * 1e6 / 1e12
        if rank == 0:
            print(json.dumps({"workload": box.name, "n": box.n, "advance": advance_step(api, ctx, db, stream, peak,
                                                                                         reps=args.steps)}))
        return

    # the step's outputs: accelerations, energy rates and both adjoints; the intermediates
    # (V, rho, A, B, dA, dB) stay in the library's kernel order
    io = api.StepIO(ctx, db, outputs=False)
    lev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(max(args.steps, 1))]

    def step(k=None, count=False):
        if k is not None:
            lev[k][0].record(stream)
        lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
        if k is not None:
            lev[k][1].record(stream)
        api.step(ctx, lv, db, io, count)
        return lv

    tuning = None
    if not args.no_tune and not args.variants and not args.launch:
        # untimed: the autotuner picks each kernel's variant on this workload's leaves
        lv_t = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
        io_t = api.StepIO(ctx, db, extras=True)
        tuning = api.autotune(ctx, lv_t, db, io_t, reps=2)
        del lv_t, io_t
        variants = {k: ctx.get_variant(k) for k in native.KERNELS}
    launch = {k: dict(zip(("persistent", "depth", "warps"), ctx.get_launch(k))) for k in native.KERNELS}
    # counting step (untimed): pair counts of every kernel
    lv_c = step(count=True)
    n_leaves = lv_c.n_leaves
    del lv_c
    torch.cuda.synchronize()
    c = io.pair_count.cpu().numpy()
    sw = io.swept_count.cpu().numpy()
    pairs = {"geometry": int(c[0]), "corrections": int(c[1]), "hydro": int(c[1]), "gravity": int(c[2]),
             "gravity_adjoint": int(c[2]), "geometry_adjoint": int(c[0])}
    # candidate pair evaluations of the forward kernels (their variants); in-range pairs / candidates
    swept = {"geometry": int(sw[0]), "hydro": int(sw[1]), "gravity": int(sw[2])}
    useful = {k: (pairs[k] / v if v else None) for k, v in swept.items()}
    pairs_step = sum(pairs.values())
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = ctypes_launches(ctx)
    ctx.check(native.lib().crk_step_profile(ctx.handle, args.steps))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for k in range(args.steps):
        step(k)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    launches = ctypes_launches(ctx) - launches0
    ms = t0.elapsed_time(t1)
    import ctypes as _ct
    prof = (_ct.c_float * 7)()
    nprof = _ct.c_int(0)
    ctx.check(native.lib().crk_step_profile_read(ctx.handle, prof, _ct.byref(nprof)))
    ctx.check(native.lib().crk_step_profile(ctx.handle, 0))
    per_stage = {"leaves": sum(lev[k][0].elapsed_time(lev[k][1]) for k in range(args.steps)) / args.steps}
    for i, s_ in enumerate(STAGES[1:]):
        per_stage[s_] = float(prof[i])
    per_stage["outputs"] = float(prof[6])
    t_max, total_pairs = aggregate(ms, pairs_step * args.steps, dist, f"cuda:{local}")
    value = total_pairs / (t_max * 1e-3)

    if args.trace_leaves:
        native.lib().crk_set_trace(ctx.handle, 1)
        api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
        native.lib().crk_set_trace(ctx.handle, 0)

    # end to end through the public API: every step's inputs are copied from pinned host memory
    # and its conservation sums read back to pinned host memory.  The copies run on a second
    # stream into one of two device input sets, so step k+1's upload overlaps step k's kernels
    # (double buffering, as an application streaming boxes through the GPU would run it).
    import copy as _copy

    keys = ("x", "y", "z", "species", "m", "h", "u", "v3")
    host = {k: getattr(db, k).cpu().pin_memory() for k in keys}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    db2 = _copy.copy(db)
    for k in keys:
        setattr(db2, k, torch.empty_like(getattr(db, k)))
    dbs = [db, db2]
    ios = [io, api.StepIO(ctx, db2, outputs=False)]
    outs = [torch.empty(4, dtype=torch.float64).pin_memory() for _ in range(2)]
    cs = torch.cuda.Stream(device=local)
    ready = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    te0, te1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    te0.record(stream)

    def upload(j):
        with torch.cuda.stream(cs):
            cs.wait_event(te0)
            cs.wait_event(freed[j])  # the previous step on this buffer has consumed its inputs
            for k in keys:
                getattr(dbs[j], k).copy_(host[k], non_blocking=True)
            ready[j].record(cs)

    upload(0)
    for i in range(e2e_steps):
        j = i % 2
        if i + 1 < e2e_steps:
            upload(1 - j)
        stream.wait_event(ready[j])
        lv_e = api.build_leaves(ctx, dbs[j].x, dbs[j].y, dbs[j].z, dbs[j].species, dbs[j].h, dbs[j].L, dbs[j].lp)
        api.step(ctx, lv_e, dbs[j], ios[j])
        outs[j].copy_(ios[j].cons, non_blocking=True)
        freed[j].record(stream)
    te1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = te0.elapsed_time(te1) / e2e_steps
    e2e_value = pairs_step / (e2e_ms * 1e-3) * world

    # roofline of the dominant kernel (ALU bound: FP32 FMA pipe)
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = n_sm * 128 * 2 * f_max * 1e6 / 1e12
    kern = {s: v for s, v in per_stage.items() if s in FLOPS_PER_PAIR}
    dom = max(kern, key=kern.get)
    achieved = FLOPS_PER_PAIR[dom] * pairs[dom] / (kern[dom] * 1e-3) / 1e12
    traffic = TRAFFIC.get((args.workload, dom, variants.get(dom), launch.get(dom, {}).get("depth"),
                           launch.get(dom, {}).get("warps")))
    f_med = float(peaks.get("clocks_under_load", {}).get("sm_mhz_median", f_max))
    f_run = float(clk.get("sm_mhz") or f_max)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic, "kernel": dom,
                "frac_at_clock": {f"{f_run:.0f} MHz (median during the timed steps)": achieved / (peak_tflops * f_run / f_max),
                                  f"{f_med:.0f} MHz (median under a GEMM load)": achieved / (peak_tflops * f_med / f_max)},
                "peak_basis": f"FP32 FMA: {n_sm} SMs x 128 lanes x 2 flop x {f_max:.0f} MHz (max SM clock)",
                "flops_per_pair": FLOPS_PER_PAIR[dom], "pairs_per_launch": pairs[dom],
                "ms_per_launch": kern[dom]}
    all_flops = sum(FLOPS_PER_PAIR[s] * pairs[s] for s in FLOPS_PER_PAIR)
    kern_ms = sum(kern.values())

    line = {"metric": "pair interactions/s per GB300 (fwd & adjoint)", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": box.name, "n_particles": box.n, "n_gas": box.n_gas, "box": box.L,
                       "leaves": n_leaves, "max_leaf": box.max_leaf, "r_cut": box.r_cut,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs (~%.1f GB) larger than L2 (129 MB)" % (h2d / 1e9)},
            "pairs_per_step": pairs, "candidates_per_step": swept, "in_range_fraction": useful,
            "stage_ms": {k: round(v, 4) for k, v in per_stage.items()},
            "variants": variants, "launch": launch,
            "autotune_ms": tuning["ms"] if tuning else None,
            "kernels_tflops": all_flops / (kern_ms * 1e-3) / 1e12,
            "roofline": roofline, "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 32,
                    "ms_per_step": e2e_ms, "steps": e2e_steps,
                    "note": "pinned host inputs copied every step on a second stream into one of two device "
                            "input sets (upload of step k+1 overlaps step k), conservation sums read back "
                            "every step; leaf build included"}}
    if not args.no_extras:
        try:
            line["extras_chain"] = extras_chain(api, ctx, db, stream, peak_tflops)
        except Exception as e:  # reported, never silent
            line["extras_chain"] = {"error": repr(e)}
    if not args.no_advance:
        try:
            line["advance"] = advance_step(api, ctx, db, stream, peak_tflops)
        except Exception as e:  # reported, never silent
            line["advance"] = {"error": repr(e)}
    if not args.no_adjoint_chain:
        try:
            line["adjoint_chain"] = adjoint_chain(api, ctx, db, stream, peak_tflops)
        except Exception as e:  # reported, never silent
            line["adjoint_chain"] = {"error": repr(e)}
    if not args.no_batched:
        try:
            line["batched_vs_plain"] = batched_vs_plain(args, local, dist, peak_tflops)
        except Exception as e:  # reported, never silent
            line["batched_vs_plain"] = {"error": repr(e)}
    if rank == 0 and not args.no_cpu_baseline:
        try:
            ref, sample, line["cpu_baseline"] = cpu_baseline(box)
            line["errors"] = sample_errors(api, ctx, db, box, ref, sample)
        except Exception as e:  # reported, never silent
            line.setdefault("cpu_baseline", {"value": None, "error": repr(e)})
            line["errors"] = {"error": repr(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


EXTRAS_FLOPS_PER_PAIR = {"extras": 103, "hydro_limited": 215, "hydro": 160}


def extras_chain(api, ctx, db, stream, peak_tflops, reps=3):
    """The Extras row: the whole step with the Extras chain (crk_extras after the
    corrections, crk_hydro_limited in place of crk_hydro) against the plain step,
    on the same leaves, through crk_step_profile (events on the context stream,
    mean of `reps` steps after a warm-up).  Outside the headline timed region.
    """
    import ctypes as _ct

    import torch
    from paper_2310_16122_gb300 import native

    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    out = {}
    for name, ex in (("plain", False), ("extras", True)):
        io = api.StepIO(ctx, db, outputs=False, extras=ex)
        api.step(ctx, lv, db, io, count=True)
        api.step(ctx, lv, db, io)
        torch.cuda.synchronize()
        pairs = int(io.pair_count.cpu().numpy()[1])
        ctx.check(native.lib().crk_step_profile(ctx.handle, reps))
        for _ in range(reps):
            api.step(ctx, lv, db, io)
        prof = (_ct.c_float * 7)()
        nprof = _ct.c_int(0)
        ctx.check(native.lib().crk_step_profile_read(ctx.handle, prof, _ct.byref(nprof)))
        ctx.check(native.lib().crk_step_profile(ctx.handle, 0))
        out[name] = {"corrections_interval": float(prof[1]), "hydro_interval": float(prof[2]),
                     "step": float(sum(prof))}
    ms_extras = out["extras"]["corrections_interval"] - out["plain"]["corrections_interval"]
    ms_lim = out["extras"]["hydro_interval"]
    tf = {"extras": EXTRAS_FLOPS_PER_PAIR["extras"] * pairs / (ms_extras * 1e-3) / 1e12,
          "hydro_limited": EXTRAS_FLOPS_PER_PAIR["hydro_limited"] * pairs / (ms_lim * 1e-3) / 1e12}
    return {"pairs_per_launch": pairs,
            "ms": {"extras": round(ms_extras, 4), "hydro_limited": round(ms_lim, 4),
                   "hydro": round(out["plain"]["hydro_interval"], 4),
                   "step_with_extras": round(out["extras"]["step"], 4), "step": round(out["plain"]["step"], 4)},
            "pairs_per_s": {"extras": pairs / (ms_extras * 1e-3), "hydro_limited": pairs / (ms_lim * 1e-3)},
            "tflops": tf, "frac_of_fp32_peak": {k: v / peak_tflops for k, v in tf.items()},
            "flops_per_pair": EXTRAS_FLOPS_PER_PAIR,
            "note": "crk_step with and without the Extras chain on the same leaves (kernel-order "
                    "intermediates); extras = difference of the corrections intervals, mean of %d steps" % reps}


# the limited forms (the Extras chain): limited hydro 215 less the equal-split energy term (8), plus the
# signal speed (9) or the compatible share of the work (17)
ADVANCE_FLOPS_PER_PAIR = {"hydro_accel": 216, "hydro_energy": 224}


def advance_step(api, ctx, db, stream, peak_tflops, reps=2):
    """The timestep row: the Acceleration and Energy passes alone on one leaf build, and
    whole two-stage kick-drift steps (crk_advance: two leaf builds, geometry, corrections,
    Extras, Acceleration, Energy and gravity at t^n and at the predicted state) on a copy of
    the workload, timed with CUDA events on the context stream after one warm-up step."""
    import copy

    import torch

    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    V, rho, _ = api.geometry(ctx, lv, db.m)
    A, B, gA, gB, _ = api.corrections(ctx, lv, V)
    rr, G, _ = api.extras(ctx, lv, db.m, db.v3, V, A, B, gA, gB)
    _, _, _, c = api.hydro_accel(ctx, lv, db.hp, db.m, db.v3, db.u, V, rr, A, B, gA, gB, G, count=True)
    torch.cuda.synchronize()
    pairs = int(c.cpu()[0])
    ms = {}
    for name in ("hydro_accel", "hydro_energy"):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for k in range(reps + 1):
            if k == 1:
                ev[0].record(stream)
            if name == "hydro_accel":
                api.hydro_accel(ctx, lv, db.hp, db.m, db.v3, db.u, V, rr, A, B, gA, gB, G)
            else:
                api.hydro_energy(ctx, lv, db.hp, db.m, db.v3, db.u, V, rr, A, B, gA, gB, db.v3, G)
        ev[1].record(stream)
        ev[1].synchronize()
        ms[name] = ev[0].elapsed_time(ev[1]) / reps
    lv.free()
    del V, rho, A, B, gA, gB, rr, G
    d = copy.copy(db)
    for k in ("x", "y", "z", "v3", "u"):
        setattr(d, k, getattr(db, k).clone())
    ap = api.AdvanceParams(cfl=0.25, dt_max=1.0, limited=True, gravity=True)
    cons = torch.zeros(4, dtype=torch.float64, device=db.x.device)
    api.advance(ctx, d, ap, conservation=cons)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        dt = api.advance(ctx, d, ap, conservation=cons)
    ev[1].record(stream)
    ev[1].synchronize()
    step_ms = ev[0].elapsed_time(ev[1]) / reps
    tf = {k: ADVANCE_FLOPS_PER_PAIR[k] * pairs / (ms[k] * 1e-3) / 1e12 for k in ms}
    return {"ms_per_step": round(step_ms, 3), "particles_per_s": db.n / (step_ms * 1e-3), "steps": reps,
            "dt_last": float(dt.cpu()[0]), "pairs_per_launch": pairs,
            "ms": {k: round(v, 4) for k, v in ms.items()},
            "pairs_per_s": {k: pairs / (v * 1e-3) for k, v in ms.items()},
            "tflops": tf, "frac_of_fp32_peak": {k: v / peak_tflops for k, v in tf.items()},
            "flops_per_pair": ADVANCE_FLOPS_PER_PAIR,
            "note": "crk_advance with Extras + limited viscosity and gravity (cfl 0.25), mean of %d steps "
                    "after one warm-up; each step = two leaf builds + the chain twice + four hydro passes, "
                    "in the kernel orders; ms/pairs_per_s/tflops are the passes as single C-ABI calls on "
                    "one leaf build (caller-order inputs: gathers and scatters included)" % reps}


# algorithmic FP32 work per in-range pair (FMA = 2): the corrections preparation sweep is the
# corrections forward sweep; its per-particle FP64 reverse is not counted
ADJOINT_FLOPS_PER_PAIR = {"corrections_adjoint_prep": 135, "corrections_adjoint_sweep": 400,
                          "hydro_adjoint": 480}


def adjoint_chain(api, ctx, db, stream, peak_tflops, reps=2):
    """The adjoint row: crk_hydro_adjoint and crk_corrections_adjoint (its two sweeps) as single
    C-ABI calls on one leaf build of the workload, random cotangents, CUDA events on the
    context stream, mean of `reps` calls after a warm-up; outside the headline timed region."""
    import torch

    lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
    V, rho, _ = api.geometry(ctx, lv, db.m)
    A, B, gA, gB, _ = api.corrections(ctx, lv, V)
    _, _, _, c = api.hydro(ctx, lv, db.hp, db.m, db.v3, db.u, V, rho, A, B, gA, gB, count=True)
    torch.cuda.synchronize()
    pairs = int(c.cpu()[0])
    gen = torch.Generator(device=db.x.device).manual_seed(7)
    n = db.n
    dvbar = torch.randn(3, n, device=db.x.device, generator=gen)
    dubar = torch.randn(n, device=db.x.device, generator=gen)
    ms = {}

    def timed(fn):
        fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            out = fn()
        ev[1].record(stream)
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / reps, out

    ms["hydro_adjoint"], g = timed(lambda: api.hydro_adjoint(ctx, lv, db.hp, db.m, db.v3, db.u, V, rho, A, B, gA, gB,
                                                             dvbar, dubar))
    ms["corrections_adjoint"], _ = timed(lambda: api.corrections_adjoint(ctx, lv, V, g["A"], g["B"], g["gA"],
                                                                         g["gB"]))
    # the whole chain, forward and reverse, in kernel order
    ms["chain"], _ = timed(lambda: api.hydro_chain_adjoint(ctx, lv, db, dvbar, dubar, forward=False))
    lv.free()
    fl = ADJOINT_FLOPS_PER_PAIR
    work = {"hydro_adjoint": fl["hydro_adjoint"] * pairs,
            "corrections_adjoint": (fl["corrections_adjoint_prep"] + fl["corrections_adjoint_sweep"]) * pairs}
    work["chain"] = (24 + 135 + 31) * pairs + work["hydro_adjoint"] + work["corrections_adjoint"]
    tf = {k: work[k] / (ms[k] * 1e-3) / 1e12 for k in ms}
    return {"pairs_per_launch": pairs, "ms": {k: round(v, 4) for k, v in ms.items()},
            "pairs_per_s": {k: pairs / (v * 1e-3) for k, v in ms.items()},
            "tflops": tf, "frac_of_fp32_peak": {k: v / peak_tflops for k, v in tf.items()},
            "flops_per_pair": fl,
            "note": "hydro_adjoint, corrections_adjoint: single C-ABI calls on caller-order inputs "
                    "(gathers and scatters included), random cotangents; corrections_adjoint = preparation "
                    "sweep (moments + FP64 reverse of the 3x3 step) + gradient sweep; chain = "
                    "crk_hydro_chain_adjoint, geometry -> corrections -> hydro forward and hydro -> "
                    "corrections -> geometry adjoints in kernel order (work: the forward sweeps 24 + 135, "
                    "the hydro forward is skipped, geometry adjoint 31); mean of %d calls after a warm-up" % reps}


def batched_vs_plain(args, local, dist, peak_tflops):
    """The many-box workload (96 boxes, sides log-uniform in [12, 48]): per-box plain launches
    against the batched form, the same kernels in the same launch shapes (autotuned on the batch).

    plain:   per box, a leaf build and a crk_step (separate launches);
    batched: one CUDA graph replayed per step, holding the capture-safe leaf rebuild of all boxes
             and one crk_step over all boxes (every pair kernel one launch over all boxes, in the
             tuned launch shape); also with every pair kernel persistent, and eagerly.
    Per-kernel times of the batched step come from crk_step_profile (CUDA events on the context
    stream around each stage) on eager steps in the same launch shapes; the leaf rebuild is timed
    the same way.  The roofline block is the dominant kernel's algorithmic FP32 rate against the
    FP32 peak, and the whole step's algorithmic rate (all kernels' flops / graph step time)."""
    import ctypes as _ct

    import numpy as np
    import torch

    from paper_2310_16122_gb300 import api, native, workloads as W

    t_gen = time.perf_counter()
    boxes = W.batched(args.batched_boxes)
    t_gen = time.perf_counter() - t_gen
    # a stream of its own: graph capture needs one other than the legacy default stream
    side = torch.cuda.Stream(device=f"cuda:{local}")
    with torch.cuda.stream(side):
        return _batched_vs_plain(args, local, peak_tflops, boxes, t_gen, side)


def _batched_vs_plain(args, local, peak_tflops, boxes, t_gen, side):
    import ctypes as _ct

    import numpy as np
    import torch

    from paper_2310_16122_gb300 import api, native

    ctx = api.Context(local, stream=side)
    dbs = [api.DeviceBox(b, device=f"cuda:{local}") for b in boxes]
    ios = [api.StepIO(ctx, db) for db in dbs]
    dbt = api.DeviceBatch(boxes, device=f"cuda:{local}")
    iot = api.StepIO(ctx, dbt)
    stream = ctx.stream
    tuned = None
    if not args.no_tune and not args.variants:
        lv_t = api.build_leaves_batch(ctx, dbt)
        tuned = api.tune(ctx, lv_t, dbt, api.StepIO(ctx, dbt, extras=True), reps=2)
        lv_t.free()
    shapes = {k: {"variant": ctx.get_variant(k), **dict(zip(("persistent", "depth", "warps"), ctx.get_launch(k)))}
              for k in native.KERNELS}

    def plain_step(count=False):
        for db, io in zip(dbs, ios):
            lv = api.build_leaves(ctx, db.x, db.y, db.z, db.species, db.h, db.L, db.lp)
            api.step(ctx, lv, db, io, count)

    def eager_batched_step(count=False):
        lv = api.build_leaves_batch(ctx, dbt)
        api.step(ctx, lv, dbt, iot, count)

    plain_step(count=True)
    eager_batched_step(count=True)
    torch.cuda.synchronize()
    per_kernel_pairs = {"geometry": int(iot.pair_count[0]), "corrections": int(iot.pair_count[1]),
                        "hydro": int(iot.pair_count[1]), "gravity": int(iot.pair_count[2]),
                        "gravity_adjoint": int(iot.pair_count[2]), "geometry_adjoint": int(iot.pair_count[0])}
    c = np.sum([io.pair_count.cpu().numpy() for io in ios], axis=0)
    p_plain = int(2 * (c[0] + c[1] + c[2]))
    p_batch = sum(per_kernel_pairs.values())
    # the same outputs, box by box
    same = all(torch.equal(io.acc, iot.acc[:, int(dbt.box_start[k]):int(dbt.box_start[k + 1])]) and
               torch.equal(io.dv, iot.dv[:, int(dbt.box_start[k]):int(dbt.box_start[k + 1])])
               for k, io in enumerate(ios))

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    res = {"plain": timed(plain_step), "batched_eager": timed(eager_batched_step)}
    # the batched driver: one graph of rebuild + step, tuned launch shapes, then all persistent
    lv_g = api.build_leaves_batch(ctx, dbt)
    io_g = api.StepIO(ctx, dbt, outputs=False)
    g = api.RebuildStepGraph(ctx, lv_g, dbt, io_g)
    res["batched_graph"] = timed(g.launch)
    status = lv_g.status()
    g.close()
    keep = {k: ctx.get_launch(k) for k in native.KERNELS}
    ctx.set_persistent(True)
    g = api.RebuildStepGraph(ctx, lv_g, dbt, io_g)
    res["batched_graph_persistent"] = timed(g.launch)
    status |= lv_g.status()
    g.close()
    for k, (pm, d, w) in keep.items():
        ctx.set_launch(k, pm, d, w)
    # per-kernel times of the batched step in the tuned shapes (eager, profiled), and the rebuild
    reps = max(args.steps, 1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ctx.check(native.lib().crk_step_profile(ctx.handle, reps))
    t_rebuild = 0.0
    for _ in range(reps):
        ev[0].record(stream)
        api.rebuild_leaves(ctx, lv_g, dbt)
        ev[1].record(stream)
        api.step(ctx, lv_g, dbt, io_g)
        torch.cuda.synchronize()
        t_rebuild += ev[0].elapsed_time(ev[1]) / reps
    prof = (_ct.c_float * 7)()
    nprof = _ct.c_int(0)
    ctx.check(native.lib().crk_step_profile_read(ctx.handle, prof, _ct.byref(nprof)))
    ctx.check(native.lib().crk_step_profile(ctx.handle, 0))
    stage_ms = {"leaves_rebuild": round(t_rebuild, 4)}
    for i, s_ in enumerate(STAGES[1:]):
        stage_ms[s_] = round(float(prof[i]), 4)
    stage_ms["outputs"] = round(float(prof[6]), 4)
    tf = {k: FLOPS_PER_PAIR[k] * per_kernel_pairs[k] / (stage_ms[k] * 1e-3) / 1e12 for k in FLOPS_PER_PAIR}
    dom = max(FLOPS_PER_PAIR, key=lambda k: stage_ms[k])
    all_flops = sum(FLOPS_PER_PAIR[k] * per_kernel_pairs[k] for k in FLOPS_PER_PAIR)
    best_graph = min(res["batched_graph"], res["batched_graph_persistent"])
    n_total = sum(b.n for b in boxes)
    return {"workload": f"{len(boxes)} boxes, sides 12-48 log-uniform, {n_total} particles",
            "pairs_per_step": p_batch, "pairs_equal": p_plain == p_batch, "outputs_equal": bool(same),
            "plain": {"ms_per_step": res["plain"], "value": p_plain / (res["plain"] * 1e-3),
                      "form": "per box: leaf build + crk_step (separate launches), tuned launch shapes"},
            "batched": {"ms_per_step": res["batched_graph"], "value": p_batch / (res["batched_graph"] * 1e-3),
                        "form": "one CUDA graph per step: capture-safe leaf rebuild of all boxes + one crk_step "
                                "over all boxes, tuned launch shapes", "leaves_status": status},
            "batched_persistent": {"ms_per_step": res["batched_graph_persistent"],
                                   "value": p_batch / (res["batched_graph_persistent"] * 1e-3),
                                   "form": "the same graph with every pair kernel persistent (resident blocks on every "
                                           "SM, atomic work queue)"},
            "batched_eager": {"ms_per_step": res["batched_eager"],
                              "value": p_batch / (res["batched_eager"] * 1e-3),
                              "form": "one multi-box leaf build (host reads back sizes) + one crk_step, eager"},
            "speedup": res["plain"] / best_graph,
            "launch_shapes": shapes, "tuning_ms": {k: r["ms"] for k, r in tuned.items()} if tuned else None,
            "stage_ms": stage_ms, "pairs_per_launch": per_kernel_pairs,
            "tflops": {k: round(v, 3) for k, v in tf.items()},
            "roofline": {"bound": "alu", "kernel": dom, "achieved": tf[dom], "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": tf[dom] / peak_tflops, "traffic": None,
                         "step_achieved": all_flops / (best_graph * 1e-3) / 1e12,
                         "step_frac": all_flops / (best_graph * 1e-3) / 1e12 / peak_tflops,
                         "kernels_frac": all_flops / (sum(stage_ms[k] for k in FLOPS_PER_PAIR) * 1e-3) / 1e12
                         / peak_tflops,
                         "note": "frac: dominant kernel of the batched step (eager, tuned shapes, CUDA events); "
                                 "step_frac: every kernel's algorithmic flops over the whole graph step "
                                 "(leaf rebuild included); kernels_frac: over the pair kernels' time only"},
            "generation_s": t_gen}


def ctypes_launches(ctx):
    import ctypes

    from paper_2310_16122_gb300 import native

    c = ctypes.c_int64(0)
    native.check(native.lib().crk_launch_count(ctx.handle, ctypes.byref(c)), ctx.handle)
    return int(c.value)


if __name__ == "__main__":
    main()
