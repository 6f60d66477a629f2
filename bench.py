"""Throughput benchmark of the resampling F-statistic on one GB300 (or N replicas).

Workload: the narrowband single-target search (H1 + L1, 10 days at dt = 0.5 s,
1 728 000 complex64 samples per detector, FFT 2^22, one sky position,
8192 f1dot x 4 f2dot = 32 768 templates), seeded Gaussian noise.  One step is
the whole hot path over that job: per-sky work (Sec. 3 steps iii-v) plus
steps vi-vii for all 32 768 templates, 2F written for every bin.

Printed JSON line: templates/s (value), 2F-bins/s, the dominant kernel's
HBM and FP32 rooflines, the FP64-GPU comparison path, the oracle on the
host cores, end-to-end through host buffers (e2e: 2F reduced on the device
to band maxima and 2F > 70; e2e_dense: every bin read back), further
workloads (one CUDA graph, uneven targets, 120-day search, refinement,
semi-coherent segments, interpolator costs), and clocks sampled during the
timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import config2, config3, config5, make_noise, template_grid  # noqa: E402

METRIC = "templates/s and 2F-bins/s on 1 GB300 at |d2F|<=1e-3·2F+0.02 vs plain FP64-GPU path"
UNIT = "templates/s"
WORKLOAD = ("narrowband single target: H1+L1, 10 d, dt=0.5 s, 1,728,000 c64 samples/det, "
            "FFT 2^22, 1 sky x 8192 f1dot x 4 f2dot = 32,768 templates, Dterms 8")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--templates", type=int, default=0, help="templates per step (0 = full job)")
    ap.add_argument("--chunk", type=int, default=256, help="templates per fstat_compute call")
    ap.add_argument("--fp64-templates", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-refine", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-interp", action="store_true")
    ap.add_argument("--no-semicoh", action="store_true")
    ap.add_argument("--no-skyheavy", action="store_true")
    ap.add_argument("--no-sft", action="store_true")
    ap.add_argument("--streams", type=int, default=2, help="template streams per plan (1..8)")
    ap.add_argument("--shape", default="", help="n1,ca,va,cb,vb: fixed FFT split and CTA shapes (skip autotune)")
    return ap.parse_args()


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0])]
        mx = [num(r[1]) for r in self.rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower().startswith("active")})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("fft_impl.cuh", "fstat_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2201_00451_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, length: int, c: int, v: int):
    """DRAM bytes per launch of one pass shape (FFT length, columns or rows
    per CTA, radix schedule) from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        if t.get("source_hash") != kernel_source_hash():
            return None
        for e in t["entries"]:
            if (e["kernel"], e["L"], e["c"], e["v"]) == (kernel, length, c, v):
                return float(e["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError, TypeError):
        pass
    return None


def set_shape(plan, args, stream):
    """Plan set-up for the headline workload: the FFT split and CTA shapes
    given by --shape, else the autotuner's choice."""
    if args.shape:
        n1_, ca, va, cb, vb = (int(v) for v in args.shape.split(","))
        plan.set_split(n1_)
        plan.set_cta(ca, cb, va, vb)
    else:
        plan.autotune(stream)


def reduce_max(value: float, world: int, device=None) -> float:
    """The slowest rank's number (whole-job time = max over replicas)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    v = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def make_inputs(t, rank):
    return [make_noise(t.seed + 7919 * rank, X, t.n_samples, t.sigmas[X], "c64")
            for X in range(len(t.detectors))]


# ------------------------------------------------------------- CPU oracle
def cpu_oracle_timing(t, xs, n_tmpl_total, n_sample_tmpl=2):
    """The FP64 oracle as it stands on a bounded sample: one per-sky step
    (iii-v) and ``n_sample_tmpl`` templates of steps vi-vii, extrapolated to
    the full job."""
    from oracle import resamp

    a, d = t.skies[0]
    t0 = time.perf_counter()
    prep = resamp.sky_prep(t, xs, a, d)
    t_sky = time.perf_counter() - t0
    tm = t.templates()
    times = []
    for k in range(n_sample_tmpl):
        s = time.perf_counter()
        resamp.twoF(t, prep, float(tm["f1dot"][k]), float(tm["f2dot"][k]))
        times.append(time.perf_counter() - s)
    t_tmpl = sum(times) / len(times)
    value = n_tmpl_total / (t_sky + n_tmpl_total * t_tmpl)
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 per-sky step (2 det x {t.n_samples} samples) in {t_sky:.2f} s + "
                      f"{n_sample_tmpl} templates of 2 x 2^{int(math.log2(t.n_fft))} FFTs at "
                      f"{t_tmpl:.2f} s each, extrapolated to {n_tmpl_total} templates"}, t_sky, t_tmpl


def _oracle_worker(job):
    """One host process of the all-cores oracle timing: the per-sky step,
    then templates of steps vi-vii; returns (per-sky s, [per-template s])."""
    t, xs, ks = job
    from oracle import resamp

    a, d = t.skies[0]
    s = time.perf_counter()
    prep = resamp.sky_prep(t, xs, a, d)
    t_sky = time.perf_counter() - s
    tm = t.templates()
    times = []
    for k in ks:
        s = time.perf_counter()
        resamp.twoF(t, prep, float(tm["f1dot"][k]), float(tm["f2dot"][k]))
        times.append(time.perf_counter() - s)
    return t_sky, times


def cpu_oracle_all_cores(t, xs, n_tmpl_total, n_per_worker=2):
    """The same oracle in one process per host core (spawned), all working
    at once on different templates; the job extrapolates as one per-sky step
    plus n_tmpl_total templates spread over the cores."""
    import concurrent.futures as cf
    import multiprocessing as mp

    workers = os.cpu_count() or 1
    n_t = t.n_templates
    jobs = [(t, xs, [(w * n_per_worker + i) % n_t for i in range(n_per_worker)]) for w in range(workers)]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, jobs))
    t_sky = statistics.median(r[0] for r in res)
    t_tmpl = statistics.median(x for r in res for x in r[1])
    value = n_tmpl_total / (t_sky + n_tmpl_total * t_tmpl / workers)
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} spawned processes at once, each 1 per-sky step (median {t_sky:.2f} s) + "
                      f"{n_per_worker} templates (median {t_tmpl:.2f} s each), extrapolated to "
                      f"{n_tmpl_total} templates over {workers} cores"}


# ------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    t = config2()
    xs = make_inputs(t, 0)
    from oracle import resamp

    a, d = t.skies[0]
    s = time.perf_counter()
    prep = resamp.sky_prep(t, xs, a, d)
    t_sky = time.perf_counter() - s
    tm = t.templates()
    for k in range(args.warmup):
        resamp.twoF(t, prep, float(tm["f1dot"][k]), float(tm["f2dot"][k]))
    times = []
    for k in range(args.steps):
        s = time.perf_counter()
        resamp.twoF(t, prep, float(tm["f1dot"][k]), float(tm["f2dot"][k]))
        times.append(time.perf_counter() - s)
    n = t.n_templates
    t_tmpl = sum(times) / len(times)
    value = n / (t_sky + n * t_tmpl)
    sample = (f"per-sky step once ({t_sky:.2f} s) + one template per step ({t_tmpl:.2f} s), "
              f"extrapolated to {n} templates")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": (t_sky + n * t_tmpl) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2201_00451_gb300 as pkg
    from paper_2201_00451_gb300 import build as fbuild

    torch.cuda.set_device(local_rank)
    if rank == 0:
        fbuild.build()
    if world > 1:
        torch.distributed.barrier()
    pkg.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)

    t = config2()
    xs = make_inputs(t, rank)
    tm_all = pkg.as_templates(t.templates())
    n_tmpl = args.templates or len(tm_all)
    tm = tm_all[:n_tmpl] if n_tmpl <= len(tm_all) else np.resize(tm_all, n_tmpl)
    chunk = min(args.chunk, n_tmpl)
    n_fft = t.n_fft

    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    plan.set_streams(args.streams)
    set_shape(plan, args, stream)
    out = torch.empty((chunk, n_fft), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2
    chunks = [tm[i:i + chunk] for i in range(0, n_tmpl, chunk)]

    def step():
        plan.invalidate_sky()
        for c in chunks:
            plan.compute_ptr(c, out.data_ptr(), stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    plan.sync()

    clocks = ClockSampler(local_rank)
    clocks.start()
    plan.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()                      # untimed: evict L2 between steps
        barrier()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        barrier()
    plan.sync()
    clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    stats = {k: plan.kernel_stats(k) for k in (0, 1, 2)}
    plan.set_profiling(False)
    ms = reduce_max(ms, world, dev)
    total_tmpl = n_tmpl * args.steps * world
    value = total_tmpl / (ms / 1e3)
    # per step: the per-sky kernels (setup, delay table, step iii per detector,
    # resampling, finalize), one coefficient kernel per chunk, two passes per template
    launches = args.steps * (len(chunks) + 2 * n_tmpl + 4 + len(t.detectors))

    # dominant kernel roofline (algorithmic bytes: 16 B per sample read for
    # pass A, 4 B per bin written for pass B)
    peak, peak_kind = peaks()
    n1, n2 = plan.split
    kinfo = {0: ("pass_a", 16.0 * t.n_samples), 1: ("pass_b", 4.0 * n_fft)}
    dom = max((0, 1), key=lambda k: stats[k][1])
    nl, tot = stats[dom]
    avg_s = tot / 1e3 / max(nl, 1)
    name, bytes_alg = kinfo[dom]
    achieved = bytes_alg / avg_s / 1e9
    ca, va, cb, vb = plan.cta
    shape = (n2, ca, va) if dom == 0 else (n1, cb, vb)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ncu_traffic(name, *shape), "kernel": name,
            "kernel_shape": {"L": shape[0], "c": shape[1], "v": shape[2]},
            "peak_source": peak_kind,
            "kernels_ms_per_launch": {kinfo[k][0]: stats[k][1] / max(stats[k][0], 1) for k in (0, 1)},
            "per_sky_ms": stats[2][1] / max(stats[2][0], 1),
            "path": {"bytes_per_template": 16.0 * t.n_samples + 4.0 * n_fft,
                     "achieved_GBps": (16.0 * t.n_samples + 4.0 * n_fft) * value / world / 1e9,
                     "frac": (16.0 * t.n_samples + 4.0 * n_fft) * value / world / 1e9 / peak},
            "split": [n1, n2], "cta": list(plan.cta)}
    # the FFT's arithmetic against the FP32 CUDA-core peak (5 N log2 N flops
    # per complex transform, two transforms per template; the FP32 peak is
    # SMs x 128 lanes x 2 flops x SM clock)
    props = torch.cuda.get_device_properties(dev)
    f32_peak = props.multi_processor_count * 128 * 2 * FP32_CLOCK_MHZ * 1e6 / 1e12
    flops_t = 2 * 5 * n_fft * math.log2(n_fft)
    flops_k = {0: 2 * 5 * n_fft * math.log2(n2), 1: 2 * 5 * n_fft * math.log2(n1)}
    roof["alu"] = {"unit": "TFLOP/s", "peak": f32_peak, "peak_source": "derived: SMs x 128 FP32 lanes x 2 x 2070 MHz",
                   "flops_per_template": flops_t,
                   "path_achieved": flops_t * value / world / 1e12,
                   "path_frac": flops_t * value / world / 1e12 / f32_peak,
                   "kernel_achieved": flops_k[dom] / avg_s / 1e12,
                   "kernel_frac": flops_k[dom] / avg_s / 1e12 / f32_peak}
    plan.close()

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "bins_per_s": value * n_fft,
                "tau_F_eff_s": 1.0 / (value * n_fft * len(t.detectors)),
                "config": {"workload": WORKLOAD, "templates_per_step": n_tmpl, "chunk": chunk,
                           "streams": args.streams,
                           "precision": "mixed: FP64 timing and phases, FP32 resample/FFT/2F",
                           "l2": "flushed between steps (256 MB write, untimed)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "gpu_launches": launches, "clocks": clocks.summary()}

    # the same step replayed as one CUDA graph (per-sky work + all templates)
    if rank == 0 and not args.no_graph:
        line["graph"] = graph_bench(t, xs, tm, chunk, dev, stream, args, flush)

    # batched uneven targets (different spans, bands, FFT lengths) in one graph
    if rank == 0 and not args.no_uneven:
        line["uneven_targets"] = uneven_bench(dev, stream)

    # large search (120 d, FFT 2^24, 64 skies x 16384 spindowns): a bounded slice
    if rank == 0 and not args.no_large:
        line["large_search"] = large_bench(dev, stream)

    # sky-dominated bank (many sky positions, few spindowns)
    if rank == 0 and not args.no_skyheavy:
        line["sky_heavy"] = sky_heavy_bench(t, xs, dev, stream, args)

    # step (ii): x_h from SFTs on the device, once per data set
    if rank == 0 and not args.no_sft:
        line["sft_to_xh"] = sft_bench(t, dev)

    # semi-coherent search: ten 10-day segments summed on the device
    if rank == 0 and not args.no_semicoh:
        line["semicoherent"] = semicoh_bench(dev, stream, args)

    # per-sky cost of the step-(v) interpolator variants and half-widths
    if rank == 0 and not args.no_interp:
        line["interp_cost"] = interp_cost(t, xs, tm_all, dev, stream)

    # FP64-GPU comparison path (same kernels in FP64), timed on a subset
    if rank == 0 and not args.no_fp64:
        line["fp64_gpu"] = fp64_gpu(t, xs, tm_all, args.fp64_templates, dev, stream, value)

    # differentiable refinement: 4096 candidates x 20 gradient-ascent steps
    if rank == 0 and not args.no_refine:
        line["refine"] = refine_bench(t, xs, dev)

    # end-to-end through the public API: pinned host x_h -> device, every
    # bin's 2F computed and reduced on the device (band maxima and 2F > 70,
    # the retention of Sec. 5.4), results back to pinned host memory; and the
    # same job reading back every bin's 2F (550 GB per step)
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_peaks(t, xs, tm, chunk, dev, stream, args)
        line["e2e_dense"] = e2e(t, xs, tm, chunk, dev, stream, args)

    if rank == 0 and not args.no_cpu:
        x64 = [x.astype(np.complex128) for x in xs]
        cb, _, _ = cpu_oracle_timing(t, x64, len(tm_all))
        line["cpu_baseline"] = cb
        line["cpu_baseline_all_cores"] = cpu_oracle_all_cores(t, x64, len(tm_all))
    if rank == 0:
        print(json.dumps(line), flush=True)


SEMI_SEGMENTS = 10


def semicoh_bench(dev, stream, args, n_f1=256, n_f2=2):
    """Semi-coherent search (Sec. 6): ten consecutive 10-day segments of
    H1 + L1 data (each 1 728 000 c64 samples, FFT 2^22, its own reference
    time), 1 sky x 256 f1dot x 2 f2dot templates at the global reference
    time; every step redoes the per-sky work of all segments and sums the
    segments' 2F with nearest-bin sliding into one 2^22-bin row per
    template.  Noise only (the work does not depend on the data)."""
    import dataclasses

    import torch

    import paper_2201_00451_gb300 as pkg

    t = config2()
    n_seg = t.n_samples
    plans = []
    for k in range(SEMI_SEGMENTS):
        seg = dataclasses.replace(t, t0=t.t0 + k * n_seg * t.dt, injections=(), name=f"seg{k}")
        p = pkg.FstatPlan.from_target(seg, pkg.MIXED)
        for X in range(len(t.detectors)):
            p.set_data(X, make_noise(t.seed + 101 * k, X, n_seg, t.sigmas[X], "c64"), t.sigmas[X])
        p.autotune(stream)
        plans.append(p)
    t_ref = t.t0 + (SEMI_SEGMENTS * n_seg // 2) * t.dt
    tm = pkg.as_templates(template_grid(t.skies, t.f1dots[-n_f1:], t.f2dots[:n_f2]))
    out = torch.empty((len(tm), t.n_fft), dtype=torch.float32, device=dev)

    def step():
        for p in plans:
            p.invalidate_sky()
        pkg.semicoherent(plans, tm, t_ref, out=out, stream=stream)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) * 1e-3 / args.steps
    for p in plans:
        p.close()
    return {"value": len(tm) / sec, "unit": "semi-coherent templates/s",
            "segment_evaluations_per_s": len(tm) * SEMI_SEGMENTS / sec,
            "ms_per_step": sec * 1e3,
            "workload": f"{SEMI_SEGMENTS} x 10 d segments (H1+L1, dt 0.5 s, 1,728,000 c64 samples each, "
                        f"FFT 2^22), 1 sky x {n_f1} f1dot x {n_f2} f2dot, per-sky work in every step"}


def interp_cost(t, xs, tm_all, dev, stream, reps=5):
    """Per-sky work (steps iii-v, 2 x 1 728 000 samples) in ms for each
    interpolation kernel and half-width D (the FFT passes do not depend on
    them)."""
    import torch

    import paper_2201_00451_gb300 as pkg

    names = {pkg.INTERP_TAPERED: "tapered", pkg.INTERP_UNTAPERED: "untapered",
             pkg.INTERP_PERIODIC: "periodic"}
    out = torch.empty((1, t.n_fft), dtype=torch.float32, device=dev)
    res = {}
    for kind, name in names.items():
        row = {}
        for d in (4, 8, 16, 32):
            plan = pkg.FstatPlan.from_target(t, pkg.MIXED, dterms=d, interp=kind)
            for X in range(len(t.detectors)):
                plan.set_data(X, xs[X], t.sigmas[X])
            plan.compute_ptr(tm_all[:1], out.data_ptr(), stream)
            plan.set_profiling(True)
            for _ in range(reps):
                plan.invalidate_sky()
                plan.compute_ptr(tm_all[:1], out.data_ptr(), stream)
            n, tot = plan.kernel_stats(2)
            plan.set_profiling(False)
            plan.close()
            row[f"D{d}"] = tot / max(n, 1)
        res[name] = row
    return {"unit": "ms per sky position", "per_sky_ms": res}


def fp64_gpu(t, xs, tm_all, n, dev, stream, mixed_value):
    import torch

    import paper_2201_00451_gb300 as pkg

    plan = pkg.FstatPlan.from_target(t, pkg.FP64)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    plan.autotune(stream)
    out = torch.empty((n, t.n_fft), dtype=torch.float32, device=dev)
    sub = tm_all[:n]
    plan.compute_ptr(sub[:1], out.data_ptr(), stream)   # warm-up
    plan.sync()
    plan.set_profiling(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.invalidate_sky()
    a.record(stream)
    plan.compute_ptr(sub, out.data_ptr(), stream)
    b.record(stream)
    plan.sync()
    ms = a.elapsed_time(b)
    n_sky, ms_sky = plan.kernel_stats(2)
    plan.close()
    per_t = (ms - ms_sky) / n
    total = t.n_templates
    v = total / ((ms_sky + total * per_t) / 1e3)
    return {"value": v, "unit": UNIT, "sample": f"per-sky step + {n} templates, extrapolated to {total}",
            "mixed_over_fp64": mixed_value / v}


def graph_bench(t, xs, tm, chunk, dev, stream, args, flush):
    """The bench step captured once as a CUDA graph (fstat_batch with an
    output ring of `chunk` rows) and replayed: same work, no per-kernel host
    launches and no timing events."""
    import torch

    import paper_2201_00451_gb300 as pkg

    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    plan.autotune(stream)
    out = torch.empty((chunk, t.n_fft), dtype=torch.float32, device=dev)
    batch = pkg.FstatBatch()
    batch.add(plan, tm, out, out_rows=chunk)
    batch.instantiate(stream)
    for _ in range(max(1, args.warmup - 1)):
        batch.launch(stream)
    torch.cuda.synchronize(dev)
    ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.launch(stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms += a.elapsed_time(b)
    nodes = batch.nodes
    batch.close()
    plan.close()
    return {"value": len(tm) * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps,
            "graph_nodes": nodes}


def uneven_bench(dev, stream):
    """Four targets with different spans, bands and FFT lengths (2^18..2^22,
    561..13333 templates), all in one CUDA graph; seeded noise."""
    import torch

    import paper_2201_00451_gb300 as pkg

    targets = config3()
    batch = pkg.FstatBatch()
    plans, keep = [], []
    n_tmpl = n_bins = 0
    for tg in targets:
        xs = [make_noise(tg.seed, X, tg.n_samples, tg.sigmas[X], "c64") for X in range(len(tg.detectors))]
        plan = pkg.FstatPlan.from_target(tg, pkg.MIXED)
        for X in range(len(tg.detectors)):
            plan.set_data(X, xs[X], tg.sigmas[X])
        plan.autotune(stream)
        out = torch.empty((64, tg.n_fft), dtype=torch.float32, device=dev)
        tm = tg.templates()
        batch.add(plan, tm, out, out_rows=64)
        plans.append(plan)
        keep.append(out)
        n_tmpl += len(tm)
        n_bins += len(tm) * tg.n_fft
    batch.instantiate(stream)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    batch.launch(stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b)
    nodes = batch.nodes
    batch.close()
    for p in plans:
        p.close()
    return {"value": n_tmpl / (ms / 1e3), "unit": UNIT, "bins_per_s": n_bins / (ms / 1e3),
            "targets": [{"n_samples": tg.n_samples, "n_fft": tg.n_fft, "templates": tg.n_templates,
                         "f_het": tg.f_het} for tg in targets],
            "ms": ms, "graph_nodes": nodes}


def large_bench(dev, stream, n_tmpl=2048):
    """The 120-day, 2^24-bin search timed on one sky position: per-sky work
    once plus n_tmpl spindown templates, extrapolated to the full bank of
    64 skies x 16 384 templates (per-sky work counted 64 times)."""
    import torch

    import paper_2201_00451_gb300 as pkg

    t = config5()
    xs = [make_noise(t.seed, X, t.n_samples, t.sigmas[X], "c64") for X in range(len(t.detectors))]
    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    plan.autotune(stream)
    tm = pkg.as_templates(t.templates()[:n_tmpl])
    out = torch.empty((64, t.n_fft), dtype=torch.float32, device=dev)
    chunks = [tm[i:i + 64] for i in range(0, len(tm), 64)]
    plan.compute_ptr(chunks[0][:2], out.data_ptr(), stream)
    plan.sync()
    plan.set_profiling(True)
    plan.invalidate_sky()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for c in chunks:
        plan.compute_ptr(c, out.data_ptr(), stream)
    b.record(stream)
    plan.sync()
    ms = a.elapsed_time(b)
    _, ms_sky = plan.kernel_stats(2)
    plan.close()
    per_t = (ms - ms_sky) / len(tm)
    total = t.n_templates
    job_s = (len(t.skies) * ms_sky + total * per_t) / 1e3
    return {"value": total / job_s, "unit": UNIT, "bins_per_s": total * t.n_fft / job_s,
            "sample": f"1 sky: per-sky work {ms_sky:.2f} ms + {len(tm)} templates at {per_t * 1e3:.1f} us each",
            "job_hours": job_s / 3600.0, "n_fft": t.n_fft, "n_samples": t.n_samples}


def sky_heavy_bench(t, xs, dev, stream, args, n_sky=128, n_f1=11):
    """A sky-dominated bank, shaped like the paper's pilot search (many sky
    positions, 11 spindowns each, Sec. 5.3): the 10-day two-detector data,
    128 sky positions in a 1 deg patch x 11 f1dot, per-sky work for every
    sky position in every step."""
    import torch

    import paper_2201_00451_gb300 as pkg

    rng = np.random.default_rng(77)
    a0, d0 = t.skies[0]
    skies = tuple((a0 + float(da), d0 + float(dd)) for da, dd in rng.uniform(-0.0087, 0.0087, (n_sky, 2)))
    tm = pkg.as_templates(template_grid(skies, t.f1dots[-n_f1:], t.f2dots[:1]))
    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    plan.autotune(stream)
    out = torch.empty((len(tm), t.n_fft), dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 1)):
        plan.compute_ptr(tm, out.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    plan.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.invalidate_sky()
        plan.compute_ptr(tm, out.data_ptr(), stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) * 1e-3 / args.steps
    n_sky_runs, ms_sky = plan.kernel_stats(2)
    plan.close()
    return {"value": len(tm) / sec, "unit": UNIT, "sky_positions_per_s": n_sky / sec,
            "per_sky_ms": ms_sky / max(n_sky_runs, 1),
            "workload": f"10-day H1+L1 data, {n_sky} sky positions x {n_f1} f1dot, FFT 2^22, "
                        "per-sky work for every position in every step"}


def sft_bench(t, dev, reps=3):
    """Step (ii) on the GPU for the 10-day two-detector data: 480 SFTs of
    1800 s per detector, a 2 Hz band of 3600 bins around f_h (dt = 0.5 s,
    1 728 000 samples), complex64 bins in pinned host memory (seeded complex
    Gaussian, the statistics of SFT bins of white noise).  Times
    fstat_set_sfts for both detectors: the host-to-device copy, the direct
    inverse transforms and the finiteness check."""
    import torch

    import paper_2201_00451_gb300 as pkg

    n_sft, nb, t_sft = 480, 3600, 1800.0
    q0 = int(round(t.f_het * t_sft)) - nb // 2
    bins = [torch.from_numpy(make_noise(t.seed + 31 * X, X, n_sft * nb, 1.0, "c64").reshape(n_sft, nb)).pin_memory()
            for X in range(len(t.detectors))]
    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_sfts(X, bins[X].numpy(), q0, t_sft, 2 * nb, 1.0)
    torch.cuda.synchronize(dev)
    s = time.perf_counter()
    for _ in range(reps):
        for X in range(len(t.detectors)):
            plan.set_sfts(X, bins[X].numpy(), q0, t_sft, 2 * nb, 1.0)
    torch.cuda.synchronize(dev)
    sec = (time.perf_counter() - s) / reps
    plan.close()
    return {"value": sec * 1e3, "unit": "ms per data set (2 detectors)",
            "sft_bins_per_s": len(t.detectors) * n_sft * nb / sec,
            "workload": f"{len(t.detectors)} det x {n_sft} SFTs of {t_sft:g} s, {nb}-bin band -> {n_sft * nb} samples"}


def refine_bench(t, xs, dev, n_cand=4096, steps=20):
    """Adjoint throughput: 2F + gradient evaluations of off-grid candidates
    (half a grid step around bank points) during 20 ascent steps."""
    import torch

    import paper_2201_00451_gb300 as pkg
    from paper_2201_00451_gb300 import refine as rf

    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    rng = np.random.Generator(np.random.PCG64(t.seed))
    tm = t.templates()
    pick = rng.integers(0, len(tm), n_cand)
    half = t.n_fft // 2
    f = t.freq(rng.integers(half - int(0.4 * t.n_fft), half + int(0.4 * t.n_fft), n_cand))
    scales = np.array([1.0 / t.t_span, 1.0 / t.t_span ** 2, np.radians(1.0 / 60.0), np.radians(1.0 / 60.0)])
    theta0 = np.stack([f, tm["f1dot"][pick], tm["alpha"][pick], tm["delta"][pick]], axis=1)
    theta0 = theta0 + rng.uniform(-0.5, 0.5, theta0.shape) * scales
    rf.refine(plan, theta0[:64], scales, steps=2)          # warm-up (builds sample tables)
    torch.cuda.synchronize(dev)
    s = time.perf_counter()
    _, hist = rf.refine(plan, theta0, scales, steps=steps)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - s
    plan.close()
    evals = n_cand * (steps + 1)
    return {"value": evals / el, "unit": "2F+gradient evaluations/s", "candidates": n_cand,
            "steps": steps, "seconds": el, "samples_per_eval": t.n_samples * len(t.detectors),
            "mean_2F_gain": float((hist[-1] - hist[0]).mean())}


def e2e(t, xs, tm, chunk, dev, stream, args):
    import torch

    import paper_2201_00451_gb300 as pkg

    n_fft = t.n_fft
    hx = [torch.from_numpy(x).pin_memory() for x in xs]
    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, hx[X].numpy(), t.sigmas[X])
    set_shape(plan, args, stream)       # the autotuner's choice from its in-process cache
    dbuf = [torch.empty((chunk, n_fft), dtype=torch.float32, device=dev) for _ in range(2)]
    hbuf = [torch.empty((chunk, n_fft), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    copy = torch.cuda.Stream(dev)
    done = [torch.cuda.Event() for _ in range(2)]
    chunks = [tm[i:i + chunk] for i in range(0, len(tm), chunk)]

    def step():
        for X in range(len(t.detectors)):
            plan.set_data(X, hx[X].numpy(), t.sigmas[X])   # pinned host -> device
        for i, c in enumerate(chunks):
            k = i & 1
            stream.wait_event(done[k])       # device buffer k free again
            plan.compute_ptr(c, dbuf[k].data_ptr(), stream)
            ev = torch.cuda.Event()
            ev.record(stream)
            copy.wait_event(ev)
            with torch.cuda.stream(copy):
                hbuf[k][: len(c)].copy_(dbuf[k][: len(c)], non_blocking=True)
            done[k].record(copy)
        copy.synchronize()
        stream.synchronize()

    for _ in range(1):
        step()
    torch.cuda.synchronize(dev)
    s = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - s
    plan.close()
    n = len(tm) * args.steps
    return {"value": n / el, "unit": UNIT,
            "h2d_bytes_per_step": int(sum(x.nbytes for x in xs)),
            "d2h_bytes_per_step": int(len(tm) * n_fft * 4)}


FP32_CLOCK_MHZ = 2070.0  # maximum SM clock of the GB300 (nvidia-smi clocks.max.sm)
PEAK_BANDS = 256         # band maxima per template (W = 16384 bins = 7.8 mHz at FFT 2^22, dt 0.5 s)
PEAK_THRESHOLD = 70.0    # the retention threshold of Sec. 5.4
PEAK_CAPACITY = 1 << 16


def e2e_peaks(t, xs, tm, chunk, dev, stream, args):
    """End to end through fstat_compute_peaks: per step the pinned x_h go up,
    every template's 2F is reduced on the device to 256 band maxima (value
    and bin) plus the list of 2F > 70, and those come back to pinned host
    buffers.  Also the device-only rate of the peaks mode (no copies)."""
    import torch

    import paper_2201_00451_gb300 as pkg

    hx = [torch.from_numpy(x).pin_memory() for x in xs]
    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, hx[X].numpy(), t.sigmas[X])
    set_shape(plan, args, stream)
    chunks = [(i, tm[i:i + chunk]) for i in range(0, len(tm), chunk)]
    outs = [{"count": torch.zeros(1, dtype=torch.int64, device=dev),
             "peaks": torch.empty((PEAK_CAPACITY, 4), dtype=torch.int32, device=dev)} for _ in range(2)]
    hmax = torch.empty((len(tm), PEAK_BANDS), dtype=torch.float32, pin_memory=True)
    hbin = torch.empty((len(tm), PEAK_BANDS), dtype=torch.int32, pin_memory=True)
    hcount = torch.empty(2, dtype=torch.int64, pin_memory=True)
    hpeaks = torch.empty((2, PEAK_CAPACITY, 4), dtype=torch.int32, pin_memory=True)
    copy = torch.cuda.Stream(dev)
    done = [torch.cuda.Event() for _ in range(2)]

    def step(with_copies=True):
        if with_copies:
            for X in range(len(t.detectors)):
                plan.set_data(X, hx[X].numpy(), t.sigmas[X])
        for k in range(2):
            outs[k]["count"].zero_()
        for j, (i, c) in enumerate(chunks):
            k = j & 1
            stream.wait_event(done[k])
            plan.compute_peaks(c, threshold=PEAK_THRESHOLD, n_bands=PEAK_BANDS, tmpl_offset=i,
                               out=outs[k], stream=stream)
            if with_copies:
                ev = torch.cuda.Event()
                ev.record(stream)
                copy.wait_event(ev)
                with torch.cuda.stream(copy):
                    hmax[i:i + len(c)].copy_(outs[k]["band_max"], non_blocking=True)
                    hbin[i:i + len(c)].copy_(outs[k]["band_bin"], non_blocking=True)
                done[k].record(copy)
        if with_copies:
            # the two crossing lists (each shared by every other chunk)
            ev = torch.cuda.Event()
            ev.record(stream)
            copy.wait_event(ev)
            with torch.cuda.stream(copy):
                for k in range(2):
                    hcount[k:k + 1].copy_(outs[k]["count"], non_blocking=True)
                    hpeaks[k].copy_(outs[k]["peaks"], non_blocking=True)
            copy.synchronize()
        stream.synchronize()

    step()
    torch.cuda.synchronize(dev)
    s = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - s
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(with_copies=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dev_s = e0.elapsed_time(e1) * 1e-3
    n_cross = int(hcount.sum())
    plan.close()
    n = len(tm) * args.steps
    return {"value": n / el, "unit": UNIT,
            "h2d_bytes_per_step": int(sum(x.nbytes for x in xs)),
            "d2h_bytes_per_step": int(hmax.nbytes + hbin.nbytes + hcount.nbytes + hpeaks.nbytes),
            "output": f"{PEAK_BANDS} band maxima (2F, bin) per template + list of 2F > {PEAK_THRESHOLD:g}",
            "crossings_per_step": n_cross,
            "device_value": n / dev_s}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
