"""Benchmark of the GB300 dexel offset path (one JSON line on rank 0).

Default workload (one step): the 2048 x 2048 grid of 1000 seeded primitives (groups of
nested hollow spheres, thin plates thinner than the radius, spheres, boxes, shells; up to 58
segments per column, 44.8 M segments, FP64 endpoints), dilated by a ball of radius 64 grid
spacings through the C ABI.  Metric: output dexel columns per second (2048^2 columns per
step).  Inputs are resident in HBM when the timed region starts and are larger than the L2.
The same step with FP32 endpoints (FP64 decisions) is timed beside it and both results are
checked against the FP64 oracle on sampled columns; the 512 x 512 six-offset step (k = 2, 8,
32, dilation and erosion) is reported under "offsets_512".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload single|offsets512|batched|morph4096]

With --impl reference the FP64 CPU oracle is timed instead (on the host cores, on a bounded
sample of output columns of the same workload per step).  For N > 1 (torchrun) every rank
runs its own replica of the workload (independent problems, no collective on the data path);
the line reports the whole-job rate with the max time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RADII = (2.0, 8.0, 32.0)
OPS = ("dilate", "erode")
K_MAIN = 64.0  # the 2048^2 workload's radius in grid spacings
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per S_mid piece of the 2048^2
# k = 64 dilation's kernels, from an ncu capture of the current kernels on a 128-row strip of
# the workload (rows 450-577, 108.1 M pieces; pass 1: its first and redo launches together),
# scaled to a full launch by the pieces processed (None once a kernel changed after its
# capture)
TRAFFIC_PER_PIECE = {"k_pass1l": 44.95, "k_levels": 64.43}
# instructions (smsp__inst_executed.sum) per S_mid piece from the same capture
INST_PER_PIECE = {"k_pass1l": 69.11, "k_levels": 78.53}
# issue peak: 152 SMs x 4 schedulers x 1 warp instruction per clock
ISSUE_PER_CLK = 152 * 4


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload():
    """The 2048 x 2048 grid of 1000 seeded primitives (FP64 endpoints)."""
    from synth import shapes
    return shapes.grid2048()


def workload512():
    from synth import shapes
    return shapes.grid512()


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
        fd, self.path = tempfile.mkstemp(prefix="dexel_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
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
        try:
            return self._summary()
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass

    def _summary(self):
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


def run_offsets512(args, rank, ws, steps=None, warmup=None, with_e2e=True):
    """The 512 x 512 step: six offsets (dilation and erosion at k = 2, 8, 32).  Headline: the
    stream-ordered entry point from one host thread on two streams; beside it the synchronous
    calls on two host threads with their own contexts and streams (which also give the
    end-to-end figure).  Returns the line's fields."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor

    import paper_1804_08968_gb300 as dx

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    g = workload512()
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

    for _ in range(warmup):
        step(grid)
    torch.cuda.synchronize()

    times = []
    launches = 0
    for _ in range(steps):
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
    ms_step = allmax(sum(times) / len(times), ws, device="cuda")

    # kernel and stage times from a serial pass (one context, one offset at a time)
    ctx = ctxs[0]
    ctx.set_profiling(True)
    rec = []
    for op in OPS:
        for k in RADII:
            flush.zero_()
            ctx.run(dx.DILATE if op == "dilate" else dx.ERODE, grid, k, main)
            rec.append((op, k, ctx.stage_ms(), ctx.stats(), ctx.kernel_ms()))
    ctx.set_profiling(False)
    torch.cuda.synchronize()

    # the headline: the same step queued with the stream-ordered entry point (one host thread,
    # no host synchronisation inside the step); the synchronous two-thread step beside it
    so = run_offsets512_enqueued(dx, grid, flush, steps, warmup, ws)
    sync_line = {"value": units * ws / (ms_step / 1e3), "unit": "columns/s",
                 "ms_per_step": ms_step, "gpu_launches": launches,
                 "how": f"dexel_dilate / dexel_erode (synchronous) on {ns} host threads, each "
                        f"its own context and stream: {plan}"}
    res = {"value": so["value"], "unit": "columns/s", "ms_per_step": so["ms_per_step"],
           "steps": steps, "warmup": warmup, "gpu_launches": so["gpu_launches"],
           "synchronous": sync_line,
           "workload": "512x512 grid, 200 seeded primitives (spheres/boxes/hollow shells, <=16 "
                       "segs/col), dilation+erosion at k=2,8,32 spacings, FP64",
           "columns_per_step": units, "nseg_in": g.nseg,
           "l2": "flushed (256 MiB write) before every timed step",
           "streams": so["how"],
           "kernel_ms": {f"{op}_k{int(k)}": {"pass1_window": km[0], "k_levels": km[1],
                                             "k_lgather": km[2], "smid_pack": km[3]}
                         for (op, k, _, _s, km) in rec},
           "stats": {f"{op}_k{int(k)}": {"mid_pieces": st[1], "out_segs": st[3],
                                         "max_pieces_col": st[4]}
                     for (op, k, _, st, _k) in rec}}

    if with_e2e:
        # end to end through the public API with host buffers (pinned), copies timed
        off_h = torch.from_numpy(np.asarray(g.col_off, np.int32)).pin_memory()
        z_h = torch.from_numpy(np.asarray(g.z, np.float64)).pin_memory()
        e2e_times = []
        h2d = d2h = 0
        for it in range(max(2, steps)):
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
        res["e2e"] = {"value": units * ws / e2e_s, "unit": "columns/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h}
    pool.shutdown()
    return res


def run_offsets512_enqueued(dx, grid, flush, steps, warmup, ws, ns=2):
    """The same six offsets queued with dexel_offset_enqueue from ONE host thread on ns
    streams (no host synchronisation inside a step; one at its end): the plans recorded by one
    synchronous call of each offset on one context, a workspace a stream (its offsets run one
    after the other there), the results checked against the synchronous ones."""
    import torch
    ctx = dx.Context(int(os.environ.get("LOCAL_RANK", "0")))
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(ns)]
    plan = offset_plan(ns)
    jobs, need = [], [0] * ns
    for w in range(ns):
        for op, k in plan[w]:
            code = dx.DILATE if op == "dilate" else dx.ERODE
            ref = ctx.run(code, grid, k, main)
            need[w] = max(need[w], ctx.last_required())
            cap = ref.nseg + ref.nseg // 4 + 1024
            jobs.append((w, code, k, ref,
                         torch.empty(grid.nx * grid.ny + 1, dtype=torch.int32, device="cuda"),
                         torch.empty((cap, 2), dtype=grid.z.dtype, device="cuda"),
                         torch.zeros(2, dtype=torch.int64, device="cuda")))
    wsb = [torch.empty(n, dtype=torch.uint8, device="cuda") for n in need]
    order = sorted(range(len(jobs)), key=lambda q: ([j[0] for j in jobs[:q]].count(jobs[q][0]), jobs[q][0]))

    def step():
        ev = torch.cuda.Event()
        ev.record(main)
        for st in streams:
            st.wait_event(ev)
        n = 0
        for q in order:  # (the streams' offsets interleaved: both streams get work at once)
            w, code, k, _, off, z, r = jobs[q]
            rc = ctx.enqueue(code, grid, k, wsb[w], off, z, r, streams[w])
            if rc != 0:
                raise RuntimeError(f"dexel_offset_enqueue: {rc}")
            n += ctx.last_launches
        for st in streams:
            main.wait_stream(st)
        return n

    for _ in range(max(warmup, 1)):
        step()
    torch.cuda.synchronize()
    for w, code, k, ref, off, z, r in jobs:
        rr = r.cpu().numpy()
        if rr[0] != 0 or rr[1] != ref.nseg or not torch.equal(off, ref.col_off) or \
                not torch.equal(z[: ref.nseg], ref.z):
            raise RuntimeError(f"stream-ordered offset differs from the synchronous one ({rr})")
    times, launches = [], 0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        launches += step()
        e1.record(main)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = allmax(sum(times) / len(times), ws, device="cuda")
    units = len(jobs) * grid.nx * grid.ny
    return {"value": units * ws / (ms / 1e3), "unit": "columns/s", "ms_per_step": ms,
            "gpu_launches": launches, "host_syncs_per_step": 1, "host_threads": 1,
            "how": f"six dexel_offset_enqueue calls from one host thread on {ns} streams ({plan}), "
                   "one context, a workspace a stream; results equal to the synchronous calls "
                   "(checked)"}


def kernel_roofline(name, km_ms, g, stats, fp32, peak, peak_kind, clk_mhz):
    """Roofline objects of one kernel of the 2048^2 call: HBM (algorithmic bytes over its
    CUDA-event time) and instruction issue (instructions from the ncu capture, scaled by the
    S_mid pieces, over the issue peak at the measured clock)."""
    ncol = g.nx * g.ny
    P = stats[1]
    s = 8 if fp32 else 16              # an endpoint pair
    sm = 10 if fp32 else 18            # an S_mid piece: two keys + int16 dx
    if name == "k_pass1l":
        # the input read once (pairs + column offsets), S_mid written with its per-column
        # start and count
        nbytes = s * g.nseg + 4 * (ncol + 1) + sm * P + 12 * ncol
        what = "k_pass1l (pass 1, x extrusion, one lane per output column)"
    else:
        # S_mid read once with its index
        nbytes = sm * P + 12 * ncol
        what = "k_levels (pass 2, per-source level unions of the capsule slices)"
    achieved = nbytes / (km_ms / 1e3) / 1e9
    tp = TRAFFIC_PER_PIECE.get(name)
    line = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None if tp is None else tp * P,
            "kernel": what + (", FP32 endpoints" if fp32 else ", FP64"),
            "algorithmic_bytes": nbytes, "ms_per_launch": km_ms, "peak_source": peak_kind}
    ipp = INST_PER_PIECE.get(name)
    issue = None
    if ipp is not None and clk_mhz:
        inst = ipp * P
        ach = inst / (km_ms / 1e3) / 1e9
        pk = ISSUE_PER_CLK * clk_mhz / 1e3
        issue = {"bound": "issue", "achieved": ach, "peak": pk, "unit": "G warp-instr/s",
                 "frac": ach / pk, "kernel": line["kernel"],
                 "peak_source": "152 SMs x 4 schedulers x measured median SM clock"}
    return line, issue


def sample_columns(n, count, seed):
    """Seeded output columns of an n x n grid: `count` random ones plus one full row."""
    import numpy as np
    rng = np.random.default_rng(seed)
    cols = rng.choice(n * n, min(count, n * n), replace=False)
    return np.unique(np.concatenate([cols, np.arange(n) + (n // 2) * n]))


def check_sampled(g, off, z, k, cols):
    """Max endpoint error and count mismatches of a dilation against the FP64 oracle."""
    import numpy as np

    import oracle
    ref = oracle.dilate(g, k, cols=cols)
    mx, mism = 0.0, 0
    for t, c in enumerate(cols):
        got = np.asarray(z[off[c]:off[c + 1]], np.float64)
        exp = ref.column(t)
        if got.shape != exp.shape:
            mism += 1
        elif exp.size:
            mx = max(mx, float(np.max(np.abs(got - exp))))
    return {"max_endpoint_error": mx, "count_mismatches": mism, "columns_checked": int(len(cols))}


def run_ours(args, rank, ws):
    """The 2048^2 k = 64 dilation, FP64 (the line's value) and FP32 endpoints beside it."""
    import numpy as np
    import torch

    import paper_1804_08968_gb300 as dx
    from synth import shapes

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    g64 = workload()
    g32 = shapes.to_float32(g64)
    gen_s = time.perf_counter() - t0
    n = g64.nx
    units = n * n
    k = K_MAIN
    ctx = dx.Context(dev)
    stream = torch.cuda.current_stream()
    grids = {"fp64": dx.Grid.from_synth(g64, dtype=torch.float64),
             "fp32": dx.Grid.from_synth(g32, dtype=torch.float32)}
    res = {}
    launches = 0
    barrier(ws)
    with ClockSampler(dev) as clk:
        for name in ("fp64", "fp32"):
            d = grids[name]
            for _ in range(args.warmup):
                out = ctx.run(dx.DILATE, d, k, stream)
            torch.cuda.synchronize()
            times = []
            nl = 0
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = ctx.run(dx.DILATE, d, k, stream)
                e1.record(stream)
                nl += ctx.last_launches
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            torch.cuda.synchronize()
            res[name] = {"ms": sum(times) / len(times), "launches": nl}
            if name == "fp64":
                launches = nl
            del out
    clocks = clk.summary()
    barrier(ws)
    ms64 = allmax(res["fp64"]["ms"], ws, device="cuda")
    ms32 = allmax(res["fp32"]["ms"], ws, device="cuda")

    # per-kernel device times from a serial profiled call of each mode, and the results
    # checked against the FP64 oracle on sampled columns (FP32: the same float32 input)
    ctx.set_profiling(True)
    prof = {}
    cols = sample_columns(n, args.check_cols, seed=11)
    for name, g in (("fp64", g64), ("fp32", g32)):
        out = ctx.run(dx.DILATE, grids[name], k, stream)
        torch.cuda.synchronize()
        prof[name] = {"stage_ms": ctx.stage_ms(), "kernel_ms": ctx.kernel_ms(), "stats": ctx.stats()}
        off, z = out.to_host()
        prof[name]["check"] = check_sampled(g, off, z, k, cols) if rank == 0 else None
        del out
    ctx.set_profiling(False)

    peak, peak_kind = measured_peaks()
    km = prof["fp64"]["kernel_ms"]
    names = ["k_pass1l", "k_levels"]
    dom = names[0] if km[0] >= km[1] else names[1]
    roof, issue = kernel_roofline(dom, km[0] if dom == "k_pass1l" else km[1], g64,
                                  prof["fp64"]["stats"], False, peak, peak_kind, clocks.get("sm_mhz"))
    other = names[1] if dom == names[0] else names[0]
    roof2, issue2 = kernel_roofline(other, km[0] if other == "k_pass1l" else km[1], g64,
                                    prof["fp64"]["stats"], False, peak, peak_kind, clocks.get("sm_mhz"))
    st = prof["fp64"]["stats"]
    s = 16
    call_bytes = 12 * (units + 1) + s * g64.nseg + 2 * 18 * st[1] + s * st[3]

    # end to end through the public API with host buffers: every step copies the input from
    # pinned host memory to the device, runs the call and reads the result back
    off_h = torch.from_numpy(np.asarray(g64.col_off, np.int32)).pin_memory()
    z_h = torch.from_numpy(np.asarray(g64.z, np.float64)).pin_memory()
    zo_h = torch.empty((max(st[3], 1), 2), dtype=torch.float64, pin_memory=True)
    oo_h = torch.empty(units + 1, dtype=torch.int32, pin_memory=True)
    e2e = []
    h2d = d2h = 0
    for _ in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gd = dx.Grid(n, n, g64.h, off_h.to("cuda", non_blocking=True), z_h.to("cuda", non_blocking=True))
        out = ctx.run(dx.DILATE, gd, k, stream)
        oo_h.copy_(out.col_off, non_blocking=True)
        zo = zo_h[: out.nseg] if out.nseg <= zo_h.shape[0] else torch.empty_like(out.z, device="cpu")
        zo.copy_(out.z, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
        h2d = off_h.numel() * 4 + z_h.numel() * 8
        d2h = oo_h.numel() * 4 + out.nseg * 16
        del gd, out
    e2e_s = allmax(statistics.median(e2e), ws, device="cuda")

    line = {
        "metric": "output dexel columns/s", "value": units * ws / (ms64 / 1e3), "unit": "columns/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms64,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2048x2048 grid, 1000 seeded primitives (nested hollow spheres, thin "
                               "plates, spheres, boxes, shells; <=58 segs/col), dilation by a ball "
                               "of radius k=64 spacings, FP64 endpoints",
                   "columns_per_step": units, "nseg_in": g64.nseg,
                   "max_segs_per_col": int(np.diff(g64.col_off).max()),
                   "l2": "inputs larger than L2 (717 MB of endpoints)", "parallelism": f"replica x{ws}"},
        "e2e": {"value": units * ws / e2e_s, "unit": "columns/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_issue": issue,
        "roofline_other": {"hbm": roof2, "issue": issue2},
        "hbm_call": {"algorithmic_bytes": call_bytes, "gbs": call_bytes / (ms64 / 1e3) / 1e9,
                     "frac": call_bytes / (ms64 / 1e3) / 1e9 / peak,
                     "formula": "12(N^2+1) + 16 nseg + 2*18 P + 16 M (FP64)"},
        "fp64": {"ms_per_step": ms64, "stage_ms": prof["fp64"]["stage_ms"],
                 "kernel_ms": dict(zip(["pass1_window", "k_levels", "k_lgather", "smid_pack"],
                                       prof["fp64"]["kernel_ms"])),
                 "mid_pieces": st[1], "out_segs": st[3], "error_vs_oracle": prof["fp64"]["check"]},
        "fp32": {"ms_per_step": ms32, "value": units * ws / (ms32 / 1e3),
                 "speedup_over_fp64": ms64 / ms32, "stage_ms": prof["fp32"]["stage_ms"],
                 "kernel_ms": dict(zip(["pass1_window", "k_levels", "k_lgather", "smid_pack"],
                                       prof["fp32"]["kernel_ms"])),
                 "mid_pieces": prof["fp32"]["stats"][1], "error_vs_oracle": prof["fp32"]["check"]},
        "clocks": clocks,
        "generate_s": gen_s,
    }
    del grids
    torch.cuda.empty_cache()
    if not args.no_512:
        line["offsets_512"] = run_offsets512(args, rank, ws, steps=min(args.steps, 10),
                                             warmup=max(3, min(args.warmup, 3)), with_e2e=False)
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g64, args)
        print(json.dumps(line), flush=True)


def oracle_sample(g, ncols, seed=0, k=K_MAIN):
    """Time the FP64 oracle's dilation of the workload on `ncols` seeded random output
    columns (a bounded sample of the step)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    cols = rng.choice(g.nx * g.ny, min(ncols, g.nx * g.ny), replace=False)
    t0 = time.perf_counter()
    oracle.dilate(g, k, cols=cols)
    return cols.size, time.perf_counter() - t0


def calibrated_columns(g, seconds):
    """Output columns the oracle takes about `seconds` for on this host (the probe gives every
    thread two of the oracle's 64-column work chunks, so that all cores are busy)."""
    import oracle
    n0, t0 = oracle_sample(g, 128 * oracle.default_threads(), seed=7)
    return int(min(g.nx * g.ny, max(200, n0 * seconds / max(t0, 1e-3))))


def cpu_baseline(g, args):
    import oracle
    oracle.build()
    cols = args.ref_cols or calibrated_columns(g, args.cpu_seconds)
    n, t = oracle_sample(g, cols)
    return {"value": n / t, "unit": "columns/s", "cores": oracle.default_threads(), "kind": "oracle",
            "sample": f"{n} random output columns of the 2048^2 k=64 dilation, FP64 brute-force "
                      f"gather over all columns within reach, {t:.1f} s"}


def run_reference(args, rank, ws):
    """The reference arm: the FP64 CPU oracle on the host cores, each step a bounded sample
    of output columns of the same workload (sized like the GPU arm's cpu_baseline)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    g = workload()
    cols = args.ref_cols or calibrated_columns(g, args.ref_seconds)
    for w in range(args.warmup):
        oracle_sample(g, max(50, cols // 10), seed=1 + w)
    times = []
    n_tot = 0
    for s in range(args.steps):
        n, t = oracle_sample(g, cols, seed=100 + s)
        times.append(t)
        n_tot += n
    per_col = sum(times) / n_tot
    units = g.nx * g.ny
    value = 1.0 / per_col
    line = {
        "impl": "reference", "metric": "output dexel columns/s", "value": value, "unit": "columns/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": units * per_col * 1e3, "ms_per_step_extrapolated": True,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "2048x2048 grid, 1000 seeded primitives (nested hollow spheres, thin "
                               "plates, spheres, boxes, shells; <=58 segs/col), dilation by a ball "
                               "of radius k=64 spacings, FP64 endpoints",
                   "columns_per_step": units, "nseg_in": g.nseg, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "columns/s", "cores": oracle.default_threads(),
                         "kind": "oracle",
                         "sample": f"{cols} random output columns per step ({n_tot} in all, "
                                   f"{sum(times):.1f} s); ms_per_step extrapolated to the "
                                   f"{units} columns of a step"},
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
    spec = shapes.batch256_shapes()
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


def contained(inner, outer, tol):
    """Every segment of `inner` lies within one segment of `outer` (one column's arrays), up to
    tol at each end (an erosion after a dilation recovers an end up to one rounding of
    (a - w) + w, so closing is extensive and opening anti-extensive up to that)."""
    import numpy as np
    if inner.shape[0] == 0:
        return True
    if outer.shape[0] == 0:
        return False
    q = np.searchsorted(outer[:, 0], inner[:, 0] + tol, side="right") - 1
    ok = q >= 0
    qq = np.maximum(q, 0)
    return bool(np.all(ok & (outer[qq, 1] >= inner[:, 1] - tol)))


def run_morph_workload(args):
    """The large morphology configuration: the 4096 x 4096 grid of 550 seeded spheres, boxes
    and hollow shells (61.6 M segments, <= 15 a column), closed and opened by a ball of radius
    k = 128 spacings, with FP64 endpoints and with FP32 endpoints (FP64 decisions).  Each
    offset runs in blocks of y lines so that its intermediate pieces fit the device.  Checks:
    the first stage (the dilation of the closing, the erosion of the opening) against the FP64
    oracle on sampled columns; closing extensive and opening anti-extensive on sampled
    columns; FP32 against FP64 results.  One JSON line."""
    import numpy as np
    import torch

    import oracle
    import paper_1804_08968_gb300 as dx
    from synth import shapes

    torch.cuda.set_device(0)
    k = 128.0
    t0 = time.perf_counter()
    g64 = shapes.grid4096()
    g32 = shapes.to_float32(g64)
    gen_s = time.perf_counter() - t0
    n = g64.nx
    ctx = dx.Context(0)
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(17)
    cols = rng.choice(n * n, args.check_cols, replace=False)
    res = {}
    with ClockSampler(0) as clk:
        for name, g, dt in (("fp64", g64, torch.float64), ("fp32", g32, torch.float32)):
            d = dx.Grid.from_synth(g, dtype=dt)
            res[name] = {}
            for opname, op, first in (("close", dx.CLOSE, dx.DILATE), ("open", dx.OPEN, dx.ERODE)):
                out = ctx.run(op, d, k)  # warm-up (sizes the scratch)
                torch.cuda.synchronize()
                times = []
                for _ in range(max(1, args.steps)):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    out = ctx.run(op, d, k)
                    e1.record(stream)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                st = ctx.stats()
                km = ctx.kernel_ms()
                off, z = out.to_host()
                del out
                # the first stage alone, against the oracle on sampled columns
                s1 = ctx.run(first, d, k)
                o1, z1 = s1.to_host()
                del s1
                torch.cuda.empty_cache()
                res[name][opname] = {"ms": statistics.median(times), "stats": st, "kernel_ms": km,
                                     "off": off, "z": z, "stage1": (o1, z1)}
            del d
            torch.cuda.empty_cache()
    out_line = {}
    for name, g in (("fp64", g64), ("fp32", g32)):
        for opname, first in (("close", "dilate"), ("open", "erode")):
            r = res[name][opname]
            o1, z1 = r["stage1"]
            ref = (oracle.dilate if first == "dilate" else oracle.erode)(g, k, cols=cols)
            mx, mism = 0.0, 0
            for t, c in enumerate(cols):
                got = np.asarray(z1[o1[c]:o1[c + 1]], np.float64)
                exp = ref.column(t)
                if got.shape != exp.shape:
                    mism += 1
                elif exp.size:
                    mx = max(mx, float(np.max(np.abs(got - exp))))
            ok = 0
            tol = 4e-7 if name == "fp32" else 1e-12
            for c in cols:
                inp = np.asarray(g.z[g.col_off[c]:g.col_off[c + 1]], np.float64)
                res_c = np.asarray(r["z"][r["off"][c]:r["off"][c + 1]], np.float64)
                ok += contained(inp, res_c, tol) if opname == "close" else contained(res_c, inp, tol)
            out_line[f"{name}_{opname}"] = {
                "ms": r["ms"], "value": n * n / (r["ms"] / 1e3), "out_segs": int(r["off"][-1]),
                "mid_pieces_last_stage": r["stats"][1], "blocks_of_lines": r["stats"][9],
                "kernel_ms": dict(zip(["pass1_window", "k_levels", "k_lgather", "smid_pack"],
                                      r["kernel_ms"])),
                "first_stage_vs_oracle": {"stage": first, "max_endpoint_error": mx,
                                          "count_mismatches": mism, "columns_checked": int(len(cols))},
                ("extensive_columns" if opname == "close" else "anti_extensive_columns"): int(ok)}
    # FP32 against FP64 (sampled columns)
    for opname in ("close", "open"):
        a, b = res["fp64"][opname], res["fp32"][opname]
        mx, mism = 0.0, 0
        for c in cols:
            za = np.asarray(a["z"][a["off"][c]:a["off"][c + 1]], np.float64)
            zb = np.asarray(b["z"][b["off"][c]:b["off"][c + 1]], np.float64)
            if za.shape != zb.shape:
                mism += 1
            elif za.size:
                mx = max(mx, float(np.max(np.abs(za - zb))))
        out_line[f"fp32_vs_fp64_{opname}"] = {"max_endpoint_difference": mx, "count_mismatches": mism,
                                              "speedup": a["ms"] / b["ms"]}
    tot64 = out_line["fp64_close"]["ms"] + out_line["fp64_open"]["ms"]
    line = {
        "metric": "output dexel columns/s", "value": 2 * n * n / (tot64 / 1e3), "unit": "columns/s",
        "n_gpus": 1, "steps": max(1, args.steps), "warmup": 1, "ms_per_step": tot64,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "4096x4096 grid, 550 seeded spheres/boxes/hollow shells (61.6 M "
                               "segments, <=15 segs/col), closing and opening at k=128 spacings "
                               "(a step: one closing and one opening, FP64)",
                   "nseg_in": g64.nseg, "l2": "inputs larger than L2", "parallelism": "replica x1"},
        **out_line,
        "clocks": clk.summary(),
        "generate_s": gen_s,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--streams", type=int, default=2,
                    help="host threads (each its own context and stream) the six offsets of the "
                         "512^2 step are split over")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-cols", type=int, default=0,
                    help="oracle columns per step of the reference arm / cpu_baseline "
                         "(0: calibrated to --ref-seconds / --cpu-seconds)")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--check-cols", type=int, default=2000,
                    help="random output columns (plus one full row) checked against the oracle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-512", action="store_true", help="skip the 512^2 six-offset extra")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one offset of a workload and exit (for ncu captures)")
    ap.add_argument("--profile-k", type=float, default=64.0)
    ap.add_argument("--profile-rows", type=int, default=0,
                    help="--profile-case on a strip of this many rows of the 2048^2 workload")
    ap.add_argument("--profile-row0", type=int, default=-1,
                    help="first row of the --profile-rows strip (default: centred)")
    ap.add_argument("--profile-mode", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--profile-op", choices=["dilate", "erode"], default="dilate")
    ap.add_argument("--workload", choices=["single", "offsets512", "batched", "morph4096"],
                    default="single",
                    help="single: the 2048^2 k=64 dilation (default line); offsets512: the 512^2 "
                         "six-offset step alone; batched: the 256-shape batched configuration; "
                         "morph4096: closing and opening of the 4096^2 grid at k=128")
    args = ap.parse_args()
    rank, ws = dist_init(args)
    if args.profile_case:
        run_profile_case(args)
        return
    if args.workload == "batched":
        run_batched_workload(args)
        return
    if args.workload == "morph4096":
        run_morph_workload(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, ws)
    elif args.workload == "offsets512":
        res = run_offsets512(args, rank, ws)
        if rank == 0:
            line = {"metric": "output dexel columns/s", "value": res["value"], "unit": "columns/s",
                    "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                    "config": {"workload": res["workload"], "columns_per_step": res["columns_per_step"],
                               "l2": res["l2"], "streams": res["streams"],
                               "parallelism": f"replica x{ws}"},
                    "e2e": res.get("e2e"), "gpu_launches": res["gpu_launches"],
                    "kernel_ms": res["kernel_ms"], "stats": res["stats"],
                    "synchronous": res.get("synchronous")}
            print(json.dumps(line), flush=True)
    else:
        run_ours(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_profile_case(args):
    """One offset of the 2048^2 workload (or a strip of its rows) for an ncu capture: a warm-up
    call, then the captured one."""
    import torch

    import paper_1804_08968_gb300 as dx
    from synth import shapes
    g = workload()
    if args.profile_rows:
        r = args.profile_rows
        j0 = (g.ny - r) // 2 if args.profile_row0 < 0 else min(args.profile_row0, g.ny - r)
        c0, c1 = g.col_off[j0 * g.nx], g.col_off[(j0 + r) * g.nx]
        g = shapes.DexelGrid(g.nx, r, g.h, g.col_off[j0 * g.nx:(j0 + r) * g.nx + 1] - c0, g.z[c0:c1])
    if args.profile_mode == "fp32":
        g = shapes.to_float32(g)
    grid = dx.Grid.from_synth(g, dtype=torch.float32 if args.profile_mode == "fp32" else torch.float64)
    ctx = dx.Context(0)
    fn = dx.DILATE if args.profile_op == "dilate" else dx.ERODE
    for _ in range(2):
        ctx.run(fn, grid, args.profile_k)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": True, "rows": g.ny, "k": args.profile_k,
                      "stats": ctx.stats()}), flush=True)


if __name__ == "__main__":
    main()
