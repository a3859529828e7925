"""Benchmark of the GB300 dexel offset path (one JSON line on rank 0).

Workload (one step): the 512 x 512 grid of 200 seeded primitives (spheres, boxes, hollow
shells; up to 16 segments per column, FP64 endpoints), dilated and eroded by balls of
radius 2, 8 and 32 grid spacings -- six offsets per step.  Metric: output dexel columns per
second (6 * 512^2 columns per step).  Inputs are resident in HBM when the timed region
starts; the L2 is flushed (a 256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --impl reference the FP64 CPU oracle is timed instead (on the host cores, on a bounded
sample of columns of the same workload per step).  For N > 1 (torchrun) every rank runs its
own replica of the workload (independent problems, no collective on the data path); the
line reports the whole-job rate with the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RADII = (2.0, 8.0, 32.0)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the k = 32
# dilation's kernels, from an ncu capture of the current kernels (None once they change):
# the pass-1 window kernel, and the pass-2 pair k_levels + k_lgather
TRAFFIC_K32_DILATE_PASS1 = 1_006_439_936
TRAFFIC_K32_DILATE_PASS2 = None  # k_lgather changed after its capture (1.55 GB then)
OPS = ("dilate", "erode")
N = 512
HBM_PEAK = None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload():
    from synth import shapes
    return shapes.config2()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        dist.init_process_group(backend)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def offset_plan(nstreams):
    """The six offsets of a step split over nstreams host threads (each its own context and
    stream), the most expensive first, each to the least loaded stream (cost: reach)."""
    order = sorted(((op, k) for op in OPS for k in RADII), key=lambda x: -x[1])
    plan = [[] for _ in range(nstreams)]
    load = [0.0] * nstreams
    for op, k in order:
        w = min(range(nstreams), key=lambda q: load[q])
        plan[w].append((op, k))
        load[w] += 1.0 + k / 8.0
    return plan


def run_ours(args, rank, ws):
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor

    import paper_1804_08968_gb300 as dx

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    g = workload()
    grid = dx.Grid.from_synth(g, dtype=torch.float64)
    ns = max(1, args.streams)
    ctxs = [dx.Context(dev) for _ in range(ns)]
    streams = [torch.cuda.Stream() for _ in range(ns)]
    plan = offset_plan(ns)
    pool = ThreadPoolExecutor(ns)
    main = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    units = len(OPS) * len(RADII) * g.nx * g.ny

    pinned = {}  # (stream, offset) -> pinned host buffers for the results, reused

    def host_buf(key, t):
        b = pinned.get(key)
        if b is None or b.numel() < t.numel():
            b = torch.empty(t.numel() + t.numel() // 8 + 64, dtype=t.dtype, pin_memory=True)
            pinned[key] = b
        return b[: t.numel()].view(t.shape)

    def worker(w, gd, fetch):
        """Stream w's offsets through the public API (each call synchronises its stream);
        fetch: copy every result to pinned host memory (asynchronous on the stream, waited
        for at the end)."""
        launches, nbytes = 0, 0
        with torch.cuda.stream(streams[w]):
            for q, (op, k) in enumerate(plan[w]):
                out = ctxs[w].run(dx.DILATE if op == "dilate" else dx.ERODE, gd, k, streams[w])
                launches += ctxs[w].last_launches
                if fetch:
                    h_off = host_buf((w, q, 0), out.col_off)
                    h_z = host_buf((w, q, 1), out.z)
                    h_off.copy_(out.col_off, non_blocking=True)
                    h_z.copy_(out.z, non_blocking=True)
                    nbytes += out.col_off.numel() * 4 + out.z.numel() * 8
            streams[w].synchronize()
        return launches, nbytes

    def step(gd, fetch=False):
        """One step: the six offsets, the streams started after everything queued on the main
        stream, the main stream waiting for all of them."""
        ev = torch.cuda.Event()
        ev.record(main)
        for st in streams:
            st.wait_event(ev)
        res = list(pool.map(lambda w: worker(w, gd, fetch), range(ns)))
        for st in streams:
            main.wait_stream(st)
        return sum(r[0] for r in res), sum(r[1] for r in res)

    for _ in range(args.warmup):
        step(grid)
    torch.cuda.synchronize()

    times = []
    launches = 0
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(main)
            n, _ = step(grid)
            e1.record(main)
            launches += n
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier(ws)
    ms_step = allmax(sum(times) / len(times), ws, device="cuda")
    value = units * ws / (ms_step / 1e3)

    # kernel and stage times from a serial pass (one context, one offset at a time, each
    # kernel bracketed by its own events; concurrent streams would stretch them)
    ctx = ctxs[0]
    ctx.set_profiling(True)
    rec = []
    for _ in range(2):
        rec = []
        for op in OPS:
            for k in RADII:
                flush.zero_()
                ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, grid, k, main)
                rec.append((op, k, ctx.stage_ms(), ctx.stats(), ctx.kernel_ms()))
    ctx.set_profiling(False)
    torch.cuda.synchronize()

    # roofline of the dominant kernel: the pass-1 window kernel of the k = 32 dilation (its
    # own event pair on the call's stream).  Algorithmic bytes: the input read once (16 B a
    # segment, 4 B a column offset), S_mid written (two FP64 keys + int16 dx = 18 B a piece)
    # with its per-column start + count (12 B).
    dom = [r for r in rec if r[0] == "dilate" and r[1] == 32.0]
    ncol = g.nx * g.ny
    dom_ms = sum(r[4][0] for r in dom) / len(dom)
    dom_bytes = 16 * g.nseg + 4 * (ncol + 1) + 18 * dom[0][3][1] + 12 * ncol
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    # the pass-2 pair of the same offset (k_levels + k_lgather): S_mid read once (18 B a
    # piece), pass-2 intervals written (16 B each), per-column start + count (12 B)
    p2_ms = sum(r[4][1] + r[4][2] for r in dom) / len(dom)
    p2_bytes = 18 * dom[0][3][1] + 16 * dom[0][3][2] + 12 * ncol
    p2_achieved = p2_bytes / (p2_ms / 1e3) / 1e9
    stages = [sum(r[2][q] for r in rec) for q in range(5)]
    kms = [sum(r[4][q] for r in rec) for q in range(4)]

    # end to end through the public API with host buffers (pinned), copies timed: each step
    # copies the input to the device and reads every result back
    off_h = torch.from_numpy(np.asarray(g.col_off, np.int32)).pin_memory()
    z_h = torch.from_numpy(np.asarray(g.z, np.float64)).pin_memory()
    e2e_times = []
    h2d = d2h = 0
    for it in range(max(2, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        off_d = off_h.to("cuda", non_blocking=True)
        z_d = z_h.to("cuda", non_blocking=True)
        gd = dx.Grid(g.nx, g.ny, g.h, off_d, z_d)
        b_in = off_h.numel() * 4 + z_h.numel() * 8
        _, b_out = step(gd, fetch=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        h2d, d2h = b_in, b_out
    e2e_s = allmax(statistics.median(e2e_times), ws, device="cuda")
    pool.shutdown()

    line = {
        "metric": "output dexel columns/s", "value": value, "unit": "columns/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512 grid, 200 seeded primitives (spheres/boxes/hollow shells, "
                               "<=16 segs/col), dilation+erosion at k=2,8,32 spacings, FP64",
                   "columns_per_step": units, "nseg_in": g.nseg, "l2": "flushed (256 MiB write) "
                   "before every timed step", "parallelism": f"replica x{ws}",
                   "streams": f"{ns} (the six offsets of a step on {ns} host threads, each its "
                              f"own context and stream: {plan})"},
        "e2e": {"value": units * ws / e2e_s, "unit": "columns/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_K32_DILATE_PASS1,
                     "kernel": "k_pass1l (pass 1, x extrusion, one lane per output column), "
                               "dilation k=32",
                     "algorithmic_bytes": dom_bytes, "ms_per_launch": dom_ms,
                     "peak_source": peak_kind},
        "roofline_pass2": {"bound": "hbm", "achieved": p2_achieved, "peak": peak, "unit": "GB/s",
                           "frac": p2_achieved / peak, "traffic": TRAFFIC_K32_DILATE_PASS2,
                           "kernel": "k_levels + k_lgather (pass 2, y dilation with per-piece "
                                     "radius), dilation k=32",
                           "algorithmic_bytes": p2_bytes, "ms_per_launch": p2_ms,
                           "peak_source": peak_kind},
        "serial_ms_per_step": {"validate+tables": stages[0], "pass1": stages[1], "pass2": stages[2],
                               "count+scan": stages[3], "write": stages[4],
                               "kernels": {"pass1_window": kms[0], "k_levels": kms[1],
                                           "k_lgather": kms[2], "smid_pack": kms[3]}},
        "stats": {f"{op}_k{int(k)}": {"mid_pieces": st[1], "out_segs": st[3],
                                      "max_pieces_col": st[4], "redo_cols": st[5]}
                  for (op, k, _, st, _k) in rec},
        "wall_s_timed": t_wall,
    }
    if rank == 0:
        line["clocks"] = clk.summary()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, args)
        print(json.dumps(line), flush=True)


def oracle_sample(g, cols_per_op, seed=0):
    """Time the FP64 oracle on a bounded sample of columns of every offset of the step."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    n = 0
    t = 0.0
    for op in OPS:
        for k in RADII:
            cols = rng.choice(g.nx * g.ny, cols_per_op, replace=False)
            t0 = time.perf_counter()
            (oracle.dilate if op == "dilate" else oracle.erode)(g, k, cols=cols)
            t += time.perf_counter() - t0
            n += cols.size
    return n, t


def cpu_baseline(g, args):
    import oracle
    oracle.build()
    # size the sample for about args.cpu_seconds of oracle work (bounded, same workload)
    n0, t0 = oracle_sample(g, 40, seed=7)
    cols = int(min(g.nx * g.ny, max(40, 40 * args.cpu_seconds / max(t0, 1e-3))))
    args.cpu_cols = cols
    n, t = oracle_sample(g, cols)
    return {"value": n / t, "unit": "columns/s", "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"{args.cpu_cols} random output columns per offset (6 offsets), FP64 brute-force "
                      f"gather, {t:.1f} s"}


def run_reference(args, rank, ws):
    if rank != 0:
        return
    import oracle
    oracle.build()
    g = workload()
    for _ in range(args.warmup):
        oracle_sample(g, 50, seed=1)
    times = []
    n_tot = 0
    for s in range(args.steps):
        n, t = oracle_sample(g, args.ref_cols, seed=100 + s)
        times.append(t)
        n_tot += n
    per_col = sum(times) / n_tot
    units = len(OPS) * len(RADII) * g.nx * g.ny
    value = 1.0 / per_col
    line = {
        "impl": "reference", "metric": "output dexel columns/s", "value": value, "unit": "columns/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": units * per_col * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "512x512 grid, 200 seeded primitives (spheres/boxes/hollow shells, "
                               "<=16 segs/col), dilation+erosion at k=2,8,32 spacings, FP64",
                   "columns_per_step": units, "nseg_in": g.nseg, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "columns/s", "cores": oracle.default_threads(),
                         "kind": "oracle",
                         "sample": f"{args.ref_cols} random output columns per offset per step"},
        "e2e": {"value": value, "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched_workload(args):
    """The batched configuration: 256 shapes (N log-uniform in 32..1024, 4-400 spheres and
    boxes each, own radius k ~ U[1, 48]; every 16th shape closed, the others dilated) in one
    dexel_offset_batched call per step, FP32 endpoints with FP64 decisions, against the plain
    FP64 GPU path (one single-shape call per shape).  The FP32 result's max endpoint error is
    measured against the FP64 oracle on sampled columns.  Prints one JSON line."""
    import numpy as np
    import torch

    import oracle
    import paper_1804_08968_gb300 as dx
    from synth import shapes

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    spec = shapes.config4_shapes()
    g64 = [shapes.raycast(prims, n) for (n, k, prims) in spec]
    g32 = [shapes.to_float32(g) for g in g64]
    ks = [k for (n, k, prims) in spec]
    ops = [dx.CLOSE if q % 16 == 0 else dx.DILATE for q in range(len(spec))]
    gen_s = time.perf_counter() - t0
    d32 = [dx.Grid.from_synth(g, dtype=torch.float32) for g in g32]
    d64 = [dx.Grid.from_synth(g, dtype=torch.float64) for g in g64]
    cols = sum(g.nx * g.ny for g in g64)
    ctx = dx.Context(0)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):  # includes the autotuning and the graph recording
        outs = ctx.run_batched(ops, d32, ks)
    torch.cuda.synchronize()
    times = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs = ctx.run_batched(ops, d32, ks)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    ms_b = statistics.median(times)
    # the plain FP64 GPU path: one call per shape
    for q in range(len(d64)):
        ctx.run(ops[q], d64[q], ks[q])
    torch.cuda.synchronize()
    t64 = []
    for _ in range(max(1, min(args.steps, 3))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for q in range(len(d64)):
            ctx.run(ops[q], d64[q], ks[q])
        e1.record(stream)
        e1.synchronize()
        t64.append(e0.elapsed_time(e1))
    ms_64 = statistics.median(t64)
    # FP32 error against the FP64 oracle (dilated shapes; sampled columns)
    rng = np.random.default_rng(0)
    max_err, mism, checked = 0.0, 0, 0
    for q in rng.choice(len(spec), 24, replace=False):
        if ops[q] != dx.DILATE:
            continue
        g = g32[q]
        cs = rng.choice(g.nx * g.ny, min(400, g.nx * g.ny), replace=False)
        ref = oracle.dilate(g, ks[q], cols=cs)
        off, z = outs[q].to_host()
        for t, c in enumerate(cs):
            got = z[off[c]:off[c + 1]].astype(np.float64)
            exp = ref.column(t)
            checked += 1
            if got.shape != exp.shape:
                mism += 1
            elif exp.size:
                max_err = max(max_err, float(np.max(np.abs(got - exp))))
    line = {
        "metric": "output dexel columns/s", "value": cols / (ms_b / 1e3), "unit": "columns/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched: 256 shapes, N log-uniform 32..1024, 4-400 spheres/boxes "
                               "each, k ~ U[1,48]; every 16th closed, the others dilated; FP32 "
                               "endpoints with FP64 decisions, one dexel_offset_batched call",
                   "columns_per_step": cols, "l2": "inputs 10x larger than L2",
                   "parallelism": "replica x1"},
        "fp64_single_calls": {"ms_per_step": ms_64, "value": cols / (ms_64 / 1e3),
                              "speedup_of_batched_fp32": ms_64 / ms_b},
        "fp32_error_vs_fp64_oracle": {"max_endpoint_error": max_err, "count_mismatches": mism,
                                      "columns_checked": checked},
        "clocks": clk.summary(),
        "generate_s": gen_s,
    }
    print(json.dumps(line), flush=True)


def run_precision_workload(args):
    """The precision configuration: the 2048 x 2048 grid of 1000 primitives (nested shells,
    thin plates thinner than r, spheres, boxes, shells; up to 58 segments per column),
    dilated by k = 64 spacings, in FP64 and in FP32 endpoints with FP64 decisions.  Reports
    both times and each result's max endpoint error and count mismatches against the FP64
    oracle on sampled columns (FP32: the oracle reads the same float32 input).  One JSON
    line."""
    import numpy as np
    import torch

    import oracle
    import paper_1804_08968_gb300 as dx
    from synth import shapes

    torch.cuda.set_device(0)
    k = 64.0
    t0 = time.perf_counter()
    g64 = shapes.config3()
    g32 = shapes.to_float32(g64)
    gen_s = time.perf_counter() - t0
    ctx = dx.Context(0)
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    res = {}
    with ClockSampler(0) as clk:
        for name, g, dt in (("fp64", g64, torch.float64), ("fp32", g32, torch.float32)):
            d = dx.Grid.from_synth(g, dtype=dt)
            out = ctx.run(dx.DILATE, d, k)  # warm-up (sizes the scratch)
            torch.cuda.synchronize()
            times = []
            for _ in range(max(1, min(args.steps, 3))):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = ctx.run(dx.DILATE, d, k)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            off, z = out.to_host()
            res[name] = {"ms": statistics.median(times), "stage_ms": ctx.stage_ms(),
                         "stats": ctx.stats(), "off": off, "z": z}
            del d, out
            torch.cuda.empty_cache()
    rng = np.random.default_rng(1)
    cols = np.concatenate([rng.choice(g64.nx * g64.ny, 2000, replace=False),
                           np.arange(2048) + 1024 * 2048])
    errs = {}
    for name, g in (("fp64", g64), ("fp32", g32)):
        ref = oracle.dilate(g, k, cols=cols)
        off, z = res[name]["off"], res[name]["z"]
        mx, mism = 0.0, 0
        for t, c in enumerate(cols):
            got = z[off[c]:off[c + 1]].astype(np.float64)
            exp = ref.column(t)
            if got.shape != exp.shape:
                mism += 1
            elif exp.size:
                mx = max(mx, float(np.max(np.abs(got - exp))))
        errs[name] = {"max_endpoint_error": mx, "count_mismatches": mism, "columns_checked": len(cols)}
    cols_n = g64.nx * g64.ny
    line = {
        "metric": "output dexel columns/s", "value": cols_n / (res["fp32"]["ms"] / 1e3),
        "unit": "columns/s", "n_gpus": 1, "steps": max(1, min(args.steps, 3)), "warmup": 1,
        "ms_per_step": res["fp32"]["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "2048x2048 grid, 1000 primitives (nested shells, thin plates, "
                               "spheres, boxes, shells), dilation k=64, FP32 endpoints with FP64 "
                               "decisions vs FP64", "nseg_in": g64.nseg,
                   "max_segs_per_col": int(np.diff(g64.col_off).max()),
                   "l2": "inputs larger than L2", "parallelism": "replica x1"},
        "fp64": {"ms_per_step": res["fp64"]["ms"], "value": cols_n / (res["fp64"]["ms"] / 1e3),
                 "stage_ms": res["fp64"]["stage_ms"], "mid_pieces": res["fp64"]["stats"][1],
                 "error_vs_oracle": errs["fp64"]},
        "fp32": {"stage_ms": res["fp32"]["stage_ms"], "mid_pieces": res["fp32"]["stats"][1],
                 "error_vs_oracle": errs["fp32"],
                 "speedup_over_fp64": res["fp64"]["ms"] / res["fp32"]["ms"]},
        "clocks": clk.summary(),
        "generate_s": gen_s,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--streams", type=int, default=2,
                    help="host threads (each its own context and stream) the six offsets of a "
                         "step are split over")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-cols", type=int, default=300)
    ap.add_argument("--ref-cols", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--profile-case", action="store_true",
                    help="run one offset of the workload and exit (for ncu captures)")
    ap.add_argument("--profile-k", type=float, default=8.0)
    ap.add_argument("--workload", choices=["single", "batched", "precision"], default="single",
                    help="batched: the 256-shape batched configuration; precision: the 2048^2 "
                         "k = 64 FP32 vs FP64 configuration (one JSON line each)")
    ap.add_argument("--profile-op", choices=["dilate", "erode"], default="dilate")
    args = ap.parse_args()
    rank, ws = dist_init(args)
    if args.profile_case:
        import torch
        import paper_1804_08968_gb300 as dx
        g = workload()
        grid = dx.Grid.from_synth(g, dtype=torch.float64)
        (dx.dilate if args.profile_op == "dilate" else dx.erode)(grid, args.profile_k)
        torch.cuda.synchronize()
        return
    if args.workload == "batched":
        run_batched_workload(args)
        return
    if args.workload == "precision":
        run_precision_workload(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
