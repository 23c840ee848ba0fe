#!/usr/bin/env python
"""DVL update throughput on B300: cells/s per alpha-TF edit.

One step = one transfer-function edit of the whole data set: the four alpha
tables change (host -> device, 4 KB) and one DVL update runs over every cell
(TF alpha per field, variation, importance, fixed-point width, device-wide
prefix scan, placement into W pixel bins, per-pixel mean and alpha).  The
once-per-data-set curve order is built before the timed region.

Workload (default): the 6-level synthetic AMR data set of ~414M cells with
4 float32 fields (128^3 base cells, logical grid 4096^3, Hilbert order),
W = 4096 pixels, P = 1, minimum importance 0.025, 256-entry TFs.  Inputs are
seeded and synthetic (they stand in for the paper's Molecular Cloud data).
The data set (~7 GB per pass) is far larger than L2, so no L2 flush is
needed between steps.

Output: one JSON line (rank 0).  Under torchrun every rank runs an
independent replica (the per-edit path needs no exchange on one GPU per data
set), timing is the max over ranks and ``value`` counts all ranks' cells.
``--impl reference`` times the CPU oracle instead (rank 0 only, a bounded
sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes.  Pass A reads the 4 float32 fields and the level byte of
# every cell and writes one u64 width total per warp step (128 cells) and one
# u64 prefix per chunk (2048 cells).  The bins stage then answers one range
# query per pixel from the value tables.  Per pixel boundary (k_bounds): the
# one 128-cell step that holds it is re-read (128 x 17 B), with its chunk's 16
# step totals (128 B), about three rounds of 32 chunk-prefix probes (768 B),
# and it writes H, S and two partial-step records of 4 fields x 24 B (201 B).
# Per pixel (k_pixels): H and S of both ends (18 B), the two records
# (192 B), two prefix-sum entries (128 B) and four sparse-table entries
# (64 B), all over the 4 fields, and the bins written (4 x 24 + 4 B).
SCAN_BYTES = 8 / 128 + 8 / 2048
BYTES_PASS_A = 4 * 4 + 1 + SCAN_BYTES
# With the kept per-cell TF entries (tables of <= 256 entries, the default)
# the width pass reads one entry byte per field and the level byte instead of
# the field values: 4 + 1 B/cell plus the totals it writes.
BYTES_PASS_A_ENT = 4 * 1 + 1 + SCAN_BYTES
BYTES_BOUNDS_PER_PIXEL = 128 * 17 + 16 * 8 + 3 * 32 * 8 + 8 + 1 + 2 * 4 * 24
BYTES_PIXELS_PER_PIXEL = 2 * 9 + 2 * 4 * 24 + 2 * 4 * 16 + 4 * 4 * 4 + 4 * 24 + 4
BYTES_BINS_PER_PIXEL = BYTES_BOUNDS_PER_PIXEL + BYTES_PIXELS_PER_PIXEL
# Value tables (once per data set and TF domain): the 4 fields read once
# (16 B/cell); per 128-cell step and field a 16-B in-block prefix and three
# 8-B (min, max) pairs written (4 x 40 / 128 B/cell); block arrays are
# 1/32 of that.
BYTES_TABLES = 4 * 4 + 4 * 40 / 128 * (1 + 1 / 32)
# with the entries: the same pass writes one entry byte per field
BYTES_TABLES_ENT = BYTES_TABLES + 4
CPU_SAMPLE_BOX = ((0, 0, 0), 32)     # 32^3 of the 128^3 base cells (1/64 of the domain)
LAUNCHES_PER_UPDATE = 5              # prepare, width pass, chunk scan, pixel bounds, pixel bins
LOG_FIELDS = (0, 2, 3)                   # dens, pres, velmag on the log10 scale
RASTER_H = 512                       # rows of the line-plot image
METRIC = "DVL update throughput (cells/s per alpha-TF edit)"


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="large")
    ap.add_argument("--width", type=int, default=4096)
    ap.add_argument("--P", type=float, default=1.0)
    ap.add_argument("--min-importance", type=float, default=0.025)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline budget (rank 0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-patterns", action="store_true",
                    help="default mode: skip the batched, served and differentiated records")
    ap.add_argument("--mode", choices=["plain", "batch", "serve", "sweep", "vmax", "diff"], default="plain",
                    help="plain: one TF edit per step (default); batch: K TFs x 4 viewports per step; "
                         "serve: Poisson TF-edit requests over 8 resident data sets; "
                         "sweep: ms/edit over the P x minimum-importance grid of the paper's Fig. 4; "
                         "vmax: exact vs approximated max V over 107 random TFs (Fig. 6); "
                         "diff: forward alpha means + adjoint gradient step of TF tuning")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="mean request arrival rate (1/s)")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="length of the request stream (s)")
    ap.add_argument("--batch-tfs", type=int, default=64)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region (read only: NVML, else nvidia-smi)
# ---------------------------------------------------------------------------

class ClockSampler:
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}
    SMI_COLS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.hw_slowdown",
                "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
                "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int):
        self.device = device
        self.samples, self.reasons, self.max_mhz, self.source = [], set(), None, None
        self._stop = threading.Event()
        self.proc = None
        try:
            import pynvml
            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByIndex(device)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
            self.source = "nvml"
        except Exception:
            self.nv = None

    def _run_nvml(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self.nv.nvmlDeviceGetClockInfo(self.h, self.nv.NVML_CLOCK_SM))
                mask = self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                self.reasons.update(k for k, b in self.BITS.items() if mask & b)
            except Exception:
                pass
            time.sleep(0.01)

    def __enter__(self):
        if self.nv:
            self.t = threading.Thread(target=self._run_nvml, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + ",".join(self.SMI_COLS),
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.lines = []
            self.t = threading.Thread(target=lambda: self.lines.extend(iter(self.proc.stdout.readline, "")),
                                      daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:   # first sample before timing
                time.sleep(0.01)
            self.skip = len(self.lines)
            self.source = "nvidia-smi"
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self.nv:
            self.t.join()
        elif self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)
            for ln in self.lines[max(self.skip - 1, 0):]:
                f = [x.strip() for x in ln.split(",")]
                if len(f) < 6:
                    continue
                try:
                    self.samples.append(float(f[0]))
                    self.max_mhz = float(f[1])
                except ValueError:
                    continue
                for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[2:6]):
                    if v.lower() == "active":
                        self.reasons.add(name)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "source": self.source}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": self.source}


# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int) -> float:
    """The maximum of a per-rank time over all ranks (the job's time): one
    all-reduce on the process group's backend (NCCL on GPUs, gloo in tests)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the
    max-over-ranks time (weak scaling: each rank holds its own data set)."""
    return units_per_rank * world / seconds


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def traffic_record():
    """dram bytes per cell of each update kernel from the committed ncu
    summary, used only while the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    import hashlib
    with open(p) as f:
        rec = json.load(f)
    src = os.path.join(ROOT, "paper_2306_11612_b300", "csrc", "update.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return rec.get("kernels", {}) if rec.get("update_cu_sha") == sha else {}


def workload_desc(amr, args, name=None):
    return {"workload": name or (f"{args.config}: {amr.meta.get('levels')}-level synthetic AMR, {amr.n} cells, "
                                 f"4 fp32 fields, Hilbert order, W={args.width}"),
            "n_cells": amr.n, "levels": amr.meta.get("levels"), "width": args.width, "P": args.P,
            "min_importance": args.min_importance, "tf_entries": 256, "fields": 4,
            "l2": "no flush: inputs (17 B/cell, ~7 GB per edit) far larger than the 126 MB L2",
            "step": "4 alpha TFs set from host + one dvl_update"}


def tf_sequence(n, seed0=1000):
    import synth
    return [synth.random_tfs(seed0 + i) for i in range(n)]


def cpu_sample(args):
    import oracle
    import synth
    amr = synth.make(args.config, box=CPU_SAMPLE_BOX) if args.config != "small" else synth.make("small")
    _, _, lev, fl = oracle.sorted_inputs(amr.lower, amr.level, amr.fields, oracle.SFC_HILBERT)
    return amr, lev, fl


def host_cores():
    """Host threads this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(amr, lev, fl, args, seconds, threads):
    """Updates of the CPU sample by the oracle on `threads` host threads
    until `seconds` have passed: (cells/s, updates, seconds)."""
    import oracle
    tfs = tf_sequence(64, 5000)
    done, i, t0 = 0, 0, time.perf_counter()
    while True:
        oracle.update(fl, lev, tfs[i % len(tfs)], P=args.P, min_importance=args.min_importance, width=args.width,
                      threads=threads)
        done += amr.n
        i += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done / el, i, el


def cpu_baseline(args, seconds):
    """The oracle, as it stands, on a bounded contiguous piece of the
    workload: on every host core (its threaded form, bit-identical to the
    sequential one) and on one core."""
    amr, lev, fl = cpu_sample(args)
    cores = host_cores()
    v_all, n_all, t_all = time_oracle(amr, lev, fl, args, seconds / 2, cores)
    v_one, n_one, t_one = time_oracle(amr, lev, fl, args, seconds / 2, 1)
    return {"value": v_all, "unit": "cells/s", "cores": cores, "kind": "oracle",
            "sample": f"{amr.n} cells = base cells {CPU_SAMPLE_BOX} of the {args.config} data set "
                      f"(a contiguous run of its curve order); {n_all} updates in {t_all:.1f} s on {cores} threads "
                      f"(orc_update_mt), {n_one} in {t_one:.1f} s on one (orc_update)",
            "one_core": {"value": v_one, "unit": "cells/s", "cores": 1}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    amr, lev, fl = cpu_sample(args)
    tfs = tf_sequence(args.steps + args.warmup)
    cores = host_cores()
    kw = dict(P=args.P, min_importance=args.min_importance, width=args.width, threads=cores)
    for i in range(args.warmup):
        oracle.update(fl, lev, tfs[i], **kw)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.update(fl, lev, tfs[args.warmup + i], **kw)
    el = time.perf_counter() - t0
    value = amr.n * args.steps / el
    name = f"{args.config} (CPU sample: base cells {CPU_SAMPLE_BOX}, {amr.n} cells), W={args.width}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
            "data": "synthetic", "config": workload_desc(amr, args, name),
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                             "sample": f"{amr.n} cells of the {args.config} data set per step, oracle on "
                                       f"{cores} host threads (orc_update_mt)"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2306_11612_b300 as dvl
    import synth

    t_gen = time.perf_counter()
    amr = synth.make(args.config, pinned=True)
    t_gen = time.perf_counter() - t_gen
    # the library's kernels run on this stream; the timing events go on it too
    stream = torch.cuda.Stream(local)
    ctx = dvl.DVL(local, stream)
    t0 = time.perf_counter()
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    t_load = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.build_order(dvl.SFC_HILBERT)
    ctx.sync()
    t_build = time.perf_counter() - t0
    tfs = tf_sequence(args.steps + args.warmup)
    kw = dict(P=args.P, min_importance=args.min_importance, width=args.width)

    # the first update also builds the value tables (once per data set and TF domain)
    t0 = time.perf_counter()
    ctx.set_tfs(tfs[0])
    ctx.update(**kw)
    ctx.sync()
    t_first = (time.perf_counter() - t0) * 1e3
    for i in range(1, args.warmup):
        ctx.set_tfs(tfs[i])
        ctx.update(**kw)
    ctx.sync()
    ctx.set_option(dvl.OPT_TIMING, 1)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            ctx.set_tfs(tfs[args.warmup + i])
            ctx.update(**kw)
            marks[i].record(stream)
        end.record(stream)
        end.synchronize()
    barrier()
    ms = start.elapsed_time(end)
    per_edit = [start.elapsed_time(marks[0])] + [marks[i - 1].elapsed_time(marks[i]) for i in range(1, args.steps)]
    tail = per_edit[20:] if len(per_edit) > 40 else per_edit
    edit_pct = {"p50_ms": statistics.median(tail),
                "p99_ms": sorted(tail)[min(len(tail) - 1, int(0.99 * len(tail)))],
                "edits": f"{len(per_edit) - len(tail)}..{len(per_edit) - 1}"}
    stages = ctx.get_timings()
    ent = bool(ctx.get_stats()["entries"])
    bytes_pass_a = BYTES_PASS_A_ENT if ent else BYTES_PASS_A
    bytes_tables = BYTES_TABLES_ENT if ent else BYTES_TABLES
    # the same edits with the width pass streaming the field values instead of
    # the kept entries (DVL_OPT_ENTRIES = 0), for comparison
    field_stream = None
    if ent:
        ctx.set_option(dvl.OPT_ENTRIES, 0)
        for i in range(2):
            ctx.set_tfs(tfs[i % len(tfs)])
            ctx.update(**kw)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(10):
            ctx.set_tfs(tfs[i % len(tfs)])
            ctx.update(**kw)
        f1.record(stream)
        f1.synchronize()
        fs = ctx.get_timings()
        field_stream = {"ms_per_edit": f0.elapsed_time(f1) / 10, "pass_a_ms": fs["pass_a"],
                        "pass_a_gbs": BYTES_PASS_A * amr.n / (fs["pass_a"] * 1e-3) / 1e9,
                        "note": "DVL_OPT_ENTRIES = 0: the width pass reads the field values (17 B/cell)"}
        ctx.set_option(dvl.OPT_ENTRIES, 1)
        ctx.set_tfs(tfs[0])
        ctx.update(**kw)
        ctx.sync()
        ctx.get_timings()
    # TF-domain edits: every field's [lo, hi] moves, so each update first
    # rebuilds the value tables (once per domain) and then runs as usual
    dlo, dhi = ctx.read_data_range()
    n_dom = 10
    doms = []
    for i in range(n_dom + 2):
        f = 0.002 * (i + 1)
        doms.append(([float(a + f * (b - a)) for a, b in zip(dlo, dhi)],
                     [float(b - f * (b - a)) for a, b in zip(dlo, dhi)]))
    for i in range(2):                                  # warm (first use of the table kernels)
        ctx.set_tfs(tfs[i % len(tfs)], lo=doms[i][0], hi=doms[i][1])
        ctx.update(**kw)
    torch.cuda.synchronize()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    d0.record(stream)
    for i in range(n_dom):
        ctx.set_tfs(tfs[i % len(tfs)], lo=doms[2 + i][0], hi=doms[2 + i][1])
        ctx.update(**kw)
    d1.record(stream)
    d1.synchronize()
    dom_wall_ms = (time.perf_counter() - t0) * 1e3 / n_dom
    dom_ms = d0.elapsed_time(d1) / n_dom
    dom_stages = ctx.get_timings()
    ctx.set_tfs(tfs[0])                                 # data-range domains again
    ctx.update(**kw)
    ctx.sync()
    ctx.set_option(dvl.OPT_TIMING, 0)
    # the line plot of the last edit (polylines of all fields, bars of one), H = 512
    img = torch.empty((2, RASTER_H, args.width), dtype=torch.uint8, device=f"cuda:{local}")
    for i in range(3):
        ctx.rasterize(RASTER_H, dvl.PLOT_Y, 0, lines=img[0], bars=img[1])
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for i in range(20):
        ctx.rasterize(RASTER_H, dvl.PLOT_Y, 0, lines=img[0], bars=img[1])
    r1.record(stream)
    r1.synchronize()
    raster_ms = r0.elapsed_time(r1) / 20
    # brushing and linking on the last edit: a pixel ROI -> cell run, key range
    # and per-cell mask (input order); then the key-range test of every cell
    mask = torch.empty(amr.n, dtype=torch.uint8, device=f"cuda:{local}")
    roi = ctx.brush(args.width // 4, args.width // 2, mask=mask)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(5):
        roi = ctx.brush(args.width // 4, args.width // 2, mask=mask)
    brush_ms = (time.perf_counter() - t0) / 5 * 1e3
    ranges = [(roi["key_first"], roi["key_last"]), (0, roi["key_first"] // 2)]
    ctx.select_keys(ranges, mask=mask)
    r0.record(stream)
    for i in range(5):
        ctx.select_keys(ranges, mask=mask)
    r1.record(stream)
    r1.synchronize()
    select_ms = r0.elapsed_time(r1) / 5
    del mask
    # per-field log10 scale of dens, pres and velmag: the one-off re-gather of
    # the values (with the scaled data ranges), the first update after it (value
    # tables rebuilt), and edits on the scaled fields
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m in LOG_FIELDS:
        ctx.set_field_scale(m, dvl.SCALE_LOG10)
    log_set_ms = (time.perf_counter() - t0) * 1e3 / len(LOG_FIELDS)
    t0 = time.perf_counter()
    ctx.update(**kw)
    ctx.sync()
    log_first_ms = (time.perf_counter() - t0) * 1e3
    r0.record(stream)
    for i in range(10):
        ctx.set_tfs(tfs[i % len(tfs)])
        ctx.update(**kw)
    r1.record(stream)
    r1.synchronize()
    log_edit_ms = r0.elapsed_time(r1) / 10
    for m in LOG_FIELDS:
        ctx.set_field_scale(m, dvl.SCALE_LINEAR)
    ctx.update(**kw)                     # value tables of the linear fields again
    ctx.sync()
    ms = max_over_ranks(ms, world)
    value = job_throughput(amr.n * args.steps, world, ms * 1e-3)

    # end to end through the public API with host buffers: TFs up, bins down
    e2e = None
    if not args.no_e2e:
        W = args.width
        # every field's bins in one call (one copy per array, one synchronisation)
        out = {k: torch.empty(W if k == "count" else 4 * W, dtype=dt, pin_memory=True).numpy() for k, dt in
               [("mean", torch.float32), ("min", torch.float32), ("max", torch.float32),
                ("y", torch.float32), ("sum", torch.float64), ("count", torch.int32)]}
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            ctx.set_tfs(tfs[args.warmup + i])
            ctx.update(**kw)
            ctx.read_bins_all(out)
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world)
        e2e = {"value": amr.n * world * args.steps / el, "unit": "cells/s",
               "h2d_bytes_per_step": 4 * 256 * 4 + 2 * 4 * 4, "d2h_bytes_per_step": 4 * W * (4 * 4 + 8) + 4 * W,
               "ms_per_step": el / args.steps * 1e3, "readback": "dvl_read_bins_all (all fields, one call)"}

    peak, peak_kind = measured_peak()
    traffic = traffic_record()
    kern = {}
    alg = {"dvl_pass_a": bytes_pass_a * amr.n, "dvl_bins": BYTES_BINS_PER_PIXEL * args.width}
    for name, key in [("dvl_pass_a", "pass_a"), ("dvl_bins", "pass_b")]:
        t_ms = stages[key]
        gbs = alg[name] / (t_ms * 1e-3) / 1e9
        kern[name] = {"ms": t_ms, "achieved_gbs": gbs, "frac": gbs / peak}
    dom = max(kern, key=lambda k: kern[k]["ms"])
    edit_bytes = alg["dvl_pass_a"] + alg["dvl_bins"]
    tr = traffic.get(dom)
    # the same kernel against the instruction issue rate (its warp
    # instructions per cell from the committed ncu capture; one instruction
    # per scheduler per clock at the sampled SM clock)
    issue_roof = None
    if tr is not None and ent and "warp_inst_per_cell" in tr:
        mhz = clk.summary().get("sm_mhz") or 2032.0
        ips = tr["warp_inst_per_cell"] * amr.n / (kern[dom]["ms"] * 1e-3)
        peak_ips = torch.cuda.get_device_properties(local).multi_processor_count * 4 * mhz * 1e6
        issue_roof = {"achieved_warp_inst_per_s": ips, "peak": peak_ips, "frac": ips / peak_ips,
                      "warp_inst_per_cell": tr["warp_inst_per_cell"], "sm_mhz": mhz}
    roofline = {"bound": "hbm", "achieved": kern[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": kern[dom]["achieved_gbs"] / peak, "kernel": dom,
                "traffic": None if tr is None else tr["dram_bytes_per_cell"] * amr.n,
                "algorithmic_bytes": alg[dom],
                "streamed": "per-cell TF entries and levels (5 B/cell)" if ent else "field values and levels (17 B/cell)",
                "issue": issue_roof,
                "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json), burst copy" if peak_kind == "measured"
                else "fallback 6.4 TB/s"}
    step_gbs = edit_bytes / (ms / args.steps * 1e-3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
            "config": workload_desc(amr, args), "roofline": roofline,
            "kernels": dict(kern, prepare_ms=stages["prepare"], finalize_ms=stages["finalize"],
                            edit_bytes_per_cell=edit_bytes / amr.n, edit_gbs=step_gbs, edit_frac=step_gbs / peak,
                            first_update_ms_with_value_tables=t_first,
                            field_stream=field_stream,
                            domain_change=dict(
                                ms_per_edit=dom_ms, wall_ms_per_edit=dom_wall_ms, edits=n_dom,
                                value_tables_ms=dom_stages["prepare"] - stages["prepare"],
                                tables_gbs=bytes_tables * amr.n / ((dom_stages["prepare"] - stages["prepare"]) * 1e-3) / 1e9,
                                tables_frac=bytes_tables * amr.n / ((dom_stages["prepare"] - stages["prepare"]) * 1e-3)
                                / 1e9 / peak,
                                note="set_tfs with new [lo, hi] for every field + dvl_update (value tables and "
                                     "per-cell TF entries rebuilt inside the update); device time by CUDA events, "
                                     "wall time on the host"),
                            rasterize_ms=raster_ms, rasterize_image=f"{RASTER_H} x {args.width}, 4 polylines + bars",
                            brush_ms=brush_ms, brush_cells=roi["n_cells"], select_keys_ms=select_ms,
                            log_scale={"fields": "dens, pres, velmag", "set_scale_ms_per_field": log_set_ms,
                                       "first_update_ms": log_first_ms, "ms_per_edit": log_edit_ms}),
            "per_edit": edit_pct,
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": LAUNCHES_PER_UPDATE * args.steps,
            "setup_s": {"generate": t_gen, "load": t_load, "build_order": t_build}}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds)
    ctx.close()
    if world == 1 and not args.no_patterns and args.config == "large":
        line.update(pattern_records(args, amr))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def pattern_records(args, full):
    """The batched, served and differentiated forms, each on its own
    configuration and next to the plain single-edit path on the same GPU, as
    compact records for the default run's line (the --mode runs print the
    full records)."""
    import copy
    import torch
    out = {}
    a = copy.copy(args)
    a.steps, a.warmup, a.no_e2e, a.no_cpu_baseline = 10, 3, True, True
    b = run_batch(a, emit=False)
    out["batch"] = {"metric": b["metric"], "value": b["value"], "unit": b["unit"], "ms_per_step": b["ms_per_step"],
                    "steps": a.steps, "config": b["config"], "roofline": b["roofline"],
                    "kernels": b["kernels"], "plain_same_gpu": b["sequential"], "clocks": b["clocks"]}
    torch.cuda.empty_cache()
    a = copy.copy(args)
    a.serve_seconds, a.warmup = 2.0, 1
    v = run_serve(a, emit=False, full=full, compare_unbatched=False)
    out["serve"] = {"metric": v["metric"], "value": v["value"], "unit": v["unit"], "p50_ms": v["p50_ms"],
                    "p99_ms": v["p99_ms"], "resident_gb": v["resident_gb"], "config": v["config"],
                    "served": v["served"], "saturated": v["saturated"], "plain_same_gpu": v["plain_closed_loop"],
                    "clocks": v["clocks"]}
    torch.cuda.empty_cache()
    a = copy.copy(args)
    a.steps, a.warmup = 20, 3
    d = run_diff(a, emit=False)
    out["diff"] = {"metric": d["metric"], "value": d["value"], "unit": d["unit"], "ms_per_step": d["ms_per_step"],
                   "steps": a.steps, "config": d["config"], "parts": d["parts"], "roofline": d["roofline"],
                   "plain_same_gpu": {"plain_update_ms": d["parts"]["plain_update_ms"],
                                      "forward_over_plain": d["parts"]["forward_ms"] / d["parts"]["plain_update_ms"]},
                   "clocks": d["clocks"]}
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# batched mode: K candidate TFs x 4 viewports per step
# ---------------------------------------------------------------------------

BATCH_WIDTHS = (512, 1024, 2048, 4096)
BATCH_METRIC = "batched DVL throughput (cells/s per (TF, viewport) bin set)"


def batch_tfs(K, seed, n_entries=256):
    import numpy as np
    import synth
    return np.stack([synth.random_tfs(seed * 100_003 + k, n_entries=n_entries) for k in range(K)])


def alg_ops_per_cell_tf(M=4):
    """Algorithmic lane operations per (cell, TF) of batched pass A: M table
    lookups, 2(M-1) min/max for the spread, the spread subtraction, three for
    the importance (scale by 1/vmax, minimum importance, level width factor),
    two for the fixed-point width (scale, round to integer) and one add."""
    return M + 2 * (M - 1) + 1 + 3 + 2 + 1


def run_batch(args, emit=True):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1 and emit:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2306_11612_b300 as dvl
    import synth

    K = args.batch_tfs
    amr = synth.make("batched", pinned=True)
    stream = torch.cuda.Stream(local)
    ctx = dvl.DVL(local, stream)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(dvl.SFC_HILBERT)
    ctx.sync()
    pairs = [(k, W) for k in range(K) for W in BATCH_WIDTHS]
    n_sets = 4
    host = [torch.from_numpy(batch_tfs(K, i)).pin_memory() for i in range(n_sets)]
    dev = [h.to(f"cuda:{local}") for h in host]
    kw = dict(P=args.P, min_importance=args.min_importance)

    t0 = time.perf_counter()
    ctx.update_batch(dev[0], pairs, **kw)          # autotune + value tables + graph capture
    ctx.sync()
    t_first = (time.perf_counter() - t0) * 1e3
    for i in range(1, max(args.warmup, 3)):
        ctx.update_batch(dev[i % n_sets], pairs, **kw)
    ctx.sync()
    cfg = ctx.batch_config()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            ctx.update_batch(dev[i % n_sets], pairs, **kw)
        end.record(stream)
        end.synchronize()
    barrier()
    ms = start.elapsed_time(end)
    replayed = ctx.batch_config()["replayed"]
    ms = max_over_ranks(ms, world)
    step_ms = ms / args.steps
    value = amr.n * len(pairs) * world / (step_ms * 1e-3)

    # per-stage device times: the same kernels as plain launches with events
    ctx.set_option(dvl.OPT_TIMING, 1)
    for i in range(min(args.steps, 20)):
        ctx.update_batch(dev[i % n_sets], pairs, **kw)
    stages = ctx.get_timings()
    ctx.set_option(dvl.OPT_TIMING, 0)

    # the same bin sets from plain single-TF updates, one after another
    host_np = [h.numpy() for h in host]
    barrier()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for k in range(K):
        ctx.set_tfs(host_np[0][k])
        for W in BATCH_WIDTHS:
            ctx.update(width=W, **kw)
    s1.record(stream)
    s1.synchronize()
    seq_ms = s0.elapsed_time(s1)
    s0.record(stream)
    for k in range(K):
        ctx.set_tfs(host_np[0][k])
        ctx.update(width=4096, **kw)
    s1.record(stream)
    s1.synchronize()
    seq64_ms = s0.elapsed_time(s1)

    # end to end: TFs from pinned host memory, every bin set back to the host
    e2e = None
    if not args.no_e2e:
        ctx.update_batch(host[0], pairs, **kw)
        nb, nc = ctx.batch_sizes()
        out = {k: torch.empty(nb, dtype=dt, pin_memory=True).numpy() for k, dt in
               [("mean", torch.float32), ("min", torch.float32), ("max", torch.float32), ("y", torch.float32),
                ("sum", torch.float64)]}
        out["count"] = torch.empty(nc, dtype=torch.int32, pin_memory=True).numpy()
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            ctx.update_batch(host[i % n_sets], pairs, **kw)
            ctx.read_batch_all(out)
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world)
        e2e = {"value": amr.n * len(pairs) * world * args.steps / el, "unit": "cells/s",
               "h2d_bytes_per_step": int(host[0].numel() * 4), "d2h_bytes_per_step": int(nb * 24 + nc * 4),
               "ms_per_step": el / args.steps * 1e3}

    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or clocks["sm_max_mhz"] or 2032
    props = torch.cuda.get_device_properties(local)
    peak_ops = props.multi_processor_count * 4 * 32 * mhz * 1e6 / 1e12     # lane-ops/s, one issue per SMSP/clk
    ops = alg_ops_per_cell_tf() * amr.n * K
    t_a = stages["pass_a"]
    achieved = ops / (t_a * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s", "frac": achieved / peak_ops,
                "traffic": None, "kernel": "dvl_pass_a_batch",
                "peak_source": f"{props.multi_processor_count} SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz "
                               "(one instruction issue per scheduler per clock)",
                "ops_per_cell_tf": alg_ops_per_cell_tf()}
    line = {"metric": BATCH_METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
            "config": {"workload": f"batched: {amr.meta.get('levels')}-level synthetic AMR, {amr.n} cells, 4 fp32 "
                                   f"fields, Hilbert order; {K} TFs x W in {list(BATCH_WIDTHS)} = {len(pairs)} "
                                   "bin sets per step",
                       "n_cells": amr.n, "tfs": K, "widths": list(BATCH_WIDTHS), "bin_sets": len(pairs),
                       "P": args.P, "min_importance": args.min_importance,
                       "l2": "no flush: cells (17 B/cell, ~0.9 GB) far larger than the 126 MB L2",
                       "step": "one dvl_update_batch (graph replay), TFs already on the device"},
            "roofline": roofline,
            "kernels": {"prepare_ms": stages["prepare"], "pass_a_batch_ms": t_a, "bins_batch_ms": stages["pass_b"],
                        "cell_tf_per_s": amr.n * K / (t_a * 1e-3), "autotuned": cfg,
                        "graph_replayed": replayed, "first_call_ms_with_tuning_and_tables": t_first},
            "sequential": {"plain_updates_same_bin_sets_ms": seq_ms,
                           "value": amr.n * len(pairs) / (seq_ms * 1e-3),
                           "speedup_batched": seq_ms / step_ms,
                           "plain_updates_64_tfs_w4096_ms": seq64_ms},
            "clocks": clocks, "e2e": e2e, "gpu_launches": 4 * args.steps}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = batch_cpu_baseline(args, K)
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1 and emit:
        torch.distributed.destroy_process_group()
    return line


def batch_cpu_baseline(args, K, seconds=None):
    """The oracle on a sub-box of the batched data set: plain updates for
    (TF, viewport) pairs until the budget is spent."""
    import oracle
    import synth
    seconds = args.cpu_seconds if seconds is None else seconds
    amr = synth.make("batched", box=CPU_SAMPLE_BOX)
    _, _, lev, fl = oracle.sorted_inputs(amr.lower, amr.level, amr.fields, oracle.SFC_HILBERT)
    tfs = batch_tfs(K, 0)
    done, t0 = 0, time.perf_counter()
    while True:
        k, W = divmod(done, len(BATCH_WIDTHS))
        oracle.update(fl, lev, tfs[k % K], P=args.P, min_importance=args.min_importance, width=BATCH_WIDTHS[W])
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": amr.n * done / el, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} plain (TF, viewport) updates of the {amr.n} cells in base cells {CPU_SAMPLE_BOX} "
                      "of the batched data set"}


# ---------------------------------------------------------------------------
# serving mode: resident data sets, Poisson TF-edit requests
# ---------------------------------------------------------------------------

SERVE_METRIC = "served DVL throughput (cells/s over TF-edit requests), p50/p99 latency"
SERVE_WIDTH = 1024


def serve_requests(n_req, rate, n_sets, M=4, seed=5):
    """Arrival times (s), data set and alpha tables of a seeded request
    stream: Poisson arrivals; each data set keeps a current TF set, 70 % of
    the requests replace one field's table, 30 % all of them."""
    import numpy as np
    import synth
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    ds = rng.integers(0, n_sets, n_req)
    state = [synth.random_tfs(900 + d, n_fields=M) for d in range(n_sets)]
    reqs = []
    for i in range(n_req):
        d = int(ds[i])
        tf = state[d].copy()
        if rng.random() < 0.7:
            tf[int(rng.integers(0, M))] = synth.random_tf(rng)
        else:
            tf = np.stack([synth.random_tf(rng) for _ in range(M)])
        state[d] = tf
        reqs.append((d, tf))
    return arrivals, reqs


def drive(srv, arrivals, reqs, width, open_loop=True):
    """Submits the stream (at its arrival times, or all at once) from one
    thread and waits for every result from another; returns wall seconds."""
    ids = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        for i, (d, tf) in enumerate(reqs):
            if open_loop:
                dt = arrivals[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
            ids[i] = srv.submit(d, tf, width)
            ready.release()

    t0 = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    for i in range(len(reqs)):
        ready.acquire()
        srv.wait(ids[i])
    th.join()
    return time.perf_counter() - t0


def overlap_ms(tl, a="run_start_ms", b="run_end_ms"):
    """From a server timeline: device time during which batches of two or
    more data sets ran at once, and the time at least one batch ran."""
    ev = []
    for r in tl:
        ev.append((float(r[a]), 1, int(r["dataset"])))
        ev.append((float(r[b]), -1, int(r["dataset"])))
    ev.sort(key=lambda e: (e[0], e[1]))
    active, last, both, busy = {}, None, 0.0, 0.0
    for t, d, ds in ev:
        if last is not None:
            live = sum(1 for c in active.values() if c > 0)
            busy += (t - last) if live >= 1 else 0.0
            both += (t - last) if live >= 2 else 0.0
        active[ds] = active.get(ds, 0) + d
        last = t
    return both, busy


def run_serve(args, emit=True, full=None, compare_unbatched=True):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1 and emit:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2306_11612_b300 as dvl
    from paper_2306_11612_b300.serve import DVLServer
    import synth

    t0 = time.perf_counter()
    sets = synth.serving_datasets(full=full)
    t_gen = time.perf_counter() - t0
    sizes = [a.n for a in sets]
    n_req = int(args.serve_rate * args.serve_seconds)
    arrivals, reqs = serve_requests(n_req, args.serve_rate, len(sets))
    kw = dict(P=args.P, min_importance=args.min_importance)

    def served(max_batch):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(local)[0]
        with DVLServer(local, max_batch=max_batch, max_inflight=len(sets), max_width=SERVE_WIDTH, **kw) as srv:
            for a in sets:
                srv.add_dataset(a.lower, a.level, a.fields)
            srv.warmup()
            torch.cuda.synchronize()
            resident = free0 - torch.cuda.mem_get_info(local)[0]
            with ClockSampler(local) as clk:
                srv.reset_stats()
                wall = drive(srv, arrivals, reqs, SERVE_WIDTH, open_loop=True)
                st = srv.stats()
                tl = srv.timeline()
                srv.reset_stats()
                wall_sat = drive(srv, arrivals, reqs, SERVE_WIDTH, open_loop=False)
                sat = srv.stats()
                tl_sat = srv.timeline()
            st["resident_gb"] = resident / 1e9
            st["overlap"] = overlap_record(tl)
            sat["overlap"] = overlap_record(tl_sat)
            return st, wall, sat, wall_sat, clk.summary()

    def overlap_record(tl):
        both, busy = overlap_ms(tl)
        ev_both, ev_busy = overlap_ms(tl, "start_ms", "end_ms")
        return {"batches": int(len(tl)), "datasets": int(len(set(tl["dataset"].tolist()))),
                "run_busy_ms": busy, "run_two_or_more_datasets_ms": both,
                "run_overlap_frac": both / busy if busy > 0 else 0.0,
                "stream_busy_ms": ev_busy, "stream_two_or_more_datasets_ms": ev_both,
                "how": "run: device clock (%globaltimer) read by each batch's first kernel at start and its last "
                       "kernel's blocks at end; stream: CUDA events around the batch's kernels on its stream"}

    st, wall, sat, wall_sat, clocks = served(64)
    if compare_unbatched:
        st1, wall1, sat1, wall_sat1, _ = served(1)
    # closed-loop plain path: one context per data set, one request at a time
    ctxs = []
    for a in sets:
        c = dvl.DVL(local)
        c.load_amr(a.lower, a.level, a.fields)
        c.build_order(dvl.SFC_HILBERT)
        ctxs.append(c)
    out = {k: np.empty((4, SERVE_WIDTH), np.float32) for k in ("mean", "min", "max", "y")}
    out["sum"] = np.empty((4, SERVE_WIDTH), np.float64)
    out["count"] = np.empty(SERVE_WIDTH, np.uint32)
    n_plain = min(n_req, 2000)
    for d, tf in reqs[:8]:                                    # warm-up
        ctxs[d].set_tfs(tf)
        ctxs[d].update(width=SERVE_WIDTH, **kw)
    lat = []
    t0 = time.perf_counter()
    for d, tf in reqs[:n_plain]:
        t1 = time.perf_counter()
        ctxs[d].set_tfs(tf)
        ctxs[d].update(width=SERVE_WIDTH, **kw)
        for m in range(4):
            ctxs[d].read_bins(m, {k: v[m] if k != "count" else v for k, v in out.items()})
        lat.append((time.perf_counter() - t1) * 1e3)
    el = time.perf_counter() - t0
    plain_cells = sum(sizes[d] for d, _ in reqs[:n_plain])
    for c in ctxs:
        c.close()

    def pick(s, wall_s):
        return {"p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"], "mean_ms": s["mean_ms"], "max_ms": s["max_ms"],
                "completed": s["completed"], "failed": s["failed"], "batches": s["batches"],
                "mean_batch": s["mean_batch"], "max_batch": s["max_batch_seen"], "cells_per_s": s["cells_per_s"],
                "requests_per_s": s["completed"] / wall_s, "wall_s": wall_s}

    pk = lambda s_, w_: dict(pick(s_, w_), overlap=s_["overlap"])
    line = {"metric": SERVE_METRIC, "value": st["cells_per_s"], "unit": "cells/s", "n_gpus": world,
            "steps": n_req, "warmup": 1, "ms_per_step": wall / n_req * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
            "config": {"workload": f"serving: {len(sets)} resident sub-boxes of the large synthetic AMR "
                                   f"({min(sizes)}..{max(sizes)} cells, {sum(sizes)} total), 4 fp32 fields; "
                                   f"Poisson TF-edit requests at {args.serve_rate:.0f}/s for "
                                   f"{args.serve_seconds:.0f} s (70 % one field, 30 % all four), W={SERVE_WIDTH}",
                       "sizes": sizes, "requests": n_req, "rate": args.serve_rate, "width": SERVE_WIDTH,
                       "max_batch": 64, "max_inflight": len(sets),
                       "step": "one request, submit to result on the host"},
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "resident_gb": st["resident_gb"],
            "served": pk(st, wall), "saturated": pk(sat, wall_sat),
            "single_request_server": ({"offered": pick(st1, wall1), "saturated": pick(sat1, wall_sat1)}
                                      if compare_unbatched else None),
            "plain_closed_loop": {"requests": n_plain, "cells_per_s": plain_cells / el,
                                  "requests_per_s": n_plain / el,
                                  "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))},
            "roofline": None, "roofline_note": "kernels as in --mode batch (pass A batch, bins)",
            "clocks": clocks, "e2e": {"value": st["cells_per_s"], "unit": "cells/s",
                                      "h2d_bytes_per_step": 4 * 256 * 4,
                                      "d2h_bytes_per_step": 4 * SERVE_WIDTH * (4 * 4 + 8) + 4 * SERVE_WIDTH},
            "setup_s": {"generate": t_gen}}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    if world > 1 and emit:
        torch.distributed.destroy_process_group()
    return line


# ---------------------------------------------------------------------------
# sweep mode: ms per edit over P and the minimum importance (Fig. 4 settings)
# ---------------------------------------------------------------------------

SWEEP_P = (0.0, 0.5, 1.0, 2.0, 5.0)
SWEEP_MIMP = (0.0, 0.025, 0.1, 0.25)


def run_sweep(args):
    import torch
    import paper_2306_11612_b300 as dvl
    import synth
    torch.cuda.set_device(0)
    amr = synth.make(args.config, pinned=True)
    stream = torch.cuda.Stream(0)
    ctx = dvl.DVL(0, stream)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(dvl.SFC_HILBERT)
    tfs = tf_sequence(args.steps + args.warmup)
    grid = []
    with ClockSampler(0) as clk:
        for P in SWEEP_P:
            for mi in SWEEP_MIMP:
                kw = dict(P=P, min_importance=mi, width=args.width)
                for i in range(args.warmup):
                    ctx.set_tfs(tfs[i])
                    ctx.update(**kw)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                for i in range(args.steps):
                    ctx.set_tfs(tfs[args.warmup + i])
                    ctx.update(**kw)
                b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b) / args.steps
                grid.append({"P": P, "min_importance": mi, "ms_per_edit": ms, "cells_per_s": amr.n / (ms * 1e-3),
                             "Q": ctx.get_stats()["Q"]})
    ctx.close()
    best = max(g["cells_per_s"] for g in grid)
    line = {"metric": METRIC + " over the P x min-importance grid", "value": min(g["cells_per_s"] for g in grid),
            "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": max(g["ms_per_edit"] for g in grid), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+u64", "data": "synthetic",
            "config": dict(workload_desc(amr, args), sweep="value = slowest setting of the grid"),
            "grid": grid, "fastest_cells_per_s": best, "clocks": clk.summary(), "roofline": None,
            "roofline_note": "per-kernel roofline in the default mode", "e2e": None,
            "gpu_launches": LAUNCHES_PER_UPDATE * args.steps * len(grid)}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# vmax mode: exact max V over the cells vs the Eq. 5/6 approximation (Fig. 6)
# ---------------------------------------------------------------------------

VMAX_TFS = 107


def run_vmax(args):
    import numpy as np
    import torch
    import paper_2306_11612_b300 as dvl
    import synth
    torch.cuda.set_device(0)
    cfg = "paper" if args.config == "large" else args.config
    amr = synth.make(cfg, pinned=True)
    stream = torch.cuda.Stream(0)
    ctx = dvl.DVL(0, stream)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(dvl.SFC_HILBERT)
    W = 1024
    tfs = tf_sequence(VMAX_TFS, seed0=5000)
    rows, t = [], {0: 0.0, 1: 0.0}
    for i, tf in enumerate(tfs):
        ctx.set_tfs(tf)
        row = {}
        for mode in (0, 1):
            ctx.update(P=args.P, min_importance=args.min_importance, width=W, vmax_mode=mode)   # warm
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.update(P=args.P, min_importance=args.min_importance, width=W, vmax_mode=mode)
            b.record(stream)
            b.synchronize()
            t[mode] += a.elapsed_time(b)
            st = ctx.get_stats()
            row["approx" if mode == 0 else "exact"] = float(st["vmax"])
            row["Q_" + ("approx" if mode == 0 else "exact")] = st["Q"]
            if mode == 0:
                cnt0 = ctx.read_bins(0)["count"].astype(np.float64)
            else:
                cnt1 = ctx.read_bins(0)["count"].astype(np.float64)
        row["count_l1"] = float(np.abs(cnt0 - cnt1).sum() / max(cnt1.sum(), 1.0))
        rows.append(row)
    ctx.close()
    ex = np.array([r["exact"] for r in rows])
    ap = np.array([r["approx"] for r in rows])
    rel = (ap - ex) / np.where(ex > 0, ex, 1.0)
    line = {"metric": "max V: Eq. 5/6 approximation vs exact maximum over cells (107 random TFs)",
            "value": float(np.median(rel)), "unit": "median relative difference (approx - exact) / exact",
            "n_gpus": 1, "steps": VMAX_TFS, "warmup": 1, "ms_per_step": (t[0] + t[1]) / VMAX_TFS,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{cfg}: {amr.n} cells, 4 fp32 fields, W={W}, {VMAX_TFS} random 8-point TFs",
                       "P": args.P, "min_importance": args.min_importance},
            "summary": {"approx_ge_exact": int((ap >= ex).sum()), "approx_lt_exact": int((ap < ex).sum()),
                        "rel_diff_min": float(rel.min()), "rel_diff_max": float(rel.max()),
                        "rel_diff_mean": float(rel.mean()),
                        "bin_count_l1_mean": float(np.mean([r["count_l1"] for r in rows])),
                        "ms_per_edit_approx": t[0] / VMAX_TFS, "ms_per_edit_exact": t[1] / VMAX_TFS},
            "per_tf": rows, "roofline": None, "e2e": None, "gpu_launches": 2 * 2 * 4 * VMAX_TFS}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# diff mode: one gradient step of automatic TF tuning (forward + adjoint)
# ---------------------------------------------------------------------------

DIFF_W, DIFF_K = 2048, 64
# algorithmic bytes per cell: the forward is one read of the cells (17 B) by
# pass A, which writes the width totals (SCAN_BYTES) and the fixed-point alpha
# sums of the 4 fields per step and per chunk; the bins come from range
# queries.  The adjoint reads the fields once more (16 B; the levels only at
# pixel crossings) with the per-pixel gradients from L2.
DIFF_FWD_BYTES = 17 + SCAN_BYTES + 4 * 8 / 128 + 4 * 8 / 2048
DIFF_FWD_BYTES_ENT = DIFF_FWD_BYTES - 4 * 3    # entries: 1 B per field instead of 4
DIFF_BWD_BYTES = 16
DIFF_BWD_BYTES_ENT = 4                          # entries: 1 B per field


def run_diff(args, emit=True):
    import numpy as np
    import torch
    import paper_2306_11612_b300 as dvl
    from paper_2306_11612_b300.diff import alpha_means
    import synth
    torch.cuda.set_device(0)
    amr = synth.make("diff", pinned=True)
    stream = torch.cuda.Stream(0)                     # the library and torch share it
    torch.cuda.set_stream(stream)
    ctx = dvl.DVL(0, stream)
    ctx.load_amr(amr.lower, amr.level, amr.fields)
    ctx.build_order(dvl.SFC_HILBERT)
    rng = np.random.default_rng(4)
    dev = torch.device("cuda:0")
    ctrl = torch.tensor(rng.uniform(0, 1, (4, DIFF_K)), dtype=torch.float32, device=dev, requires_grad=True)
    target = torch.tensor(rng.uniform(0, 1, (4, DIFF_W)), dtype=torch.float32, device=dev)
    kw = dict(width=DIFF_W, P=args.P, min_importance=args.min_importance)

    def step():
        abar = alpha_means(ctx, ctrl, **kw)
        loss = ((abar - target) ** 2).sum()
        loss.backward()
        with torch.no_grad():
            ctrl.sub_(1e-3 * ctrl.grad)
            ctrl.clamp_(0.0, 1.0)
            ctrl.grad = None
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        a.record(stream)
        for _ in range(args.steps):
            loss = step()
        b.record(stream)
        b.synchronize()
    ms = a.elapsed_time(b) / args.steps
    # the parts: forward update with alpha means, adjoint, and a plain update
    c = ctrl.detach()
    ctx.set_tf_ctrl(c, 256)
    torch.cuda.synchronize()
    parts = {}
    for name, fn in [("forward_ms", lambda: ctx.update(want_alpha=1, **kw)),
                     ("plain_update_ms", lambda: ctx.update(**kw))]:
        fn()
        a.record(stream)
        for _ in range(10):
            fn()
        b.record(stream)
        b.synchronize()
        parts[name] = a.elapsed_time(b) / 10
    ctx.update(want_alpha=1, **kw)
    g = torch.ones((4, DIFF_W), dtype=torch.float32, device=dev)
    gout = torch.empty((4, DIFF_K), dtype=torch.float32, device=dev)
    ctx.backward(g, gout)
    a.record(stream)
    for _ in range(10):
        ctx.backward(g, gout)
    b.record(stream)
    b.synchronize()
    parts["adjoint_ms"] = a.elapsed_time(b) / 10
    ctx.update(want_alpha=1, **kw)
    ent = bool(ctx.get_stats()["entries"])
    ctx.close()
    peak, _ = measured_peak()
    fwd_bytes = DIFF_FWD_BYTES_ENT if ent else DIFF_FWD_BYTES
    fwd_gbs = fwd_bytes * amr.n / (parts["forward_ms"] * 1e-3) / 1e9
    bwd_gbs = (DIFF_BWD_BYTES_ENT if ent else DIFF_BWD_BYTES) * amr.n / (parts["adjoint_ms"] * 1e-3) / 1e9
    line = {"metric": "TF-tuning gradient step (forward alpha means + adjoint), cells/s", "value": amr.n / (ms * 1e-3),
            "unit": "cells/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 gradient sums)",
            "data": "synthetic",
            "config": {"workload": f"diff: 4-level synthetic AMR, {amr.n} cells, 4 fp32 fields, {DIFF_K} control "
                                   f"points per field ({4 * DIFF_K} parameters), W={DIFF_W}, L2 loss vs a seeded target",
                       "step": "alpha_means forward, loss.backward (adjoint kernel), SGD update of the control points"},
            "parts": parts, "final_loss": float(loss.item()),
            "roofline": {"bound": "hbm", "kernel": "forward (pass A with alpha sums, range-query bins)",
                         "achieved": fwd_gbs, "peak": peak, "unit": "GB/s", "frac": fwd_gbs / peak,
                         "algorithmic_bytes_per_cell": fwd_bytes,
                         "traffic": None, "adjoint_gbs": bwd_gbs, "adjoint_frac": bwd_gbs / peak},
            "clocks": clk.summary(), "e2e": None,
            # forward: control-point tables, prepare, width pass, chunk scan, alpha-means placement,
            # finalize; adjoint: histograms, two reduction levels, chain rule
            "gpu_launches": 10 * args.steps}
    if emit:
        print(json.dumps(line), flush=True)
    torch.cuda.set_stream(torch.cuda.default_stream(0))
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "sweep":
        run_sweep(args)
    elif args.mode == "vmax":
        run_vmax(args)
    elif args.mode == "diff":
        run_diff(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
