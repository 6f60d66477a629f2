"""Throughput benchmark of the resampling F-statistic on one GB300 (or N replicas).

Headline workload: the large narrowband search (H1 + L1, 120 days at
dt = 1 s, 10 368 000 complex64 samples per detector, FFT 2^24, a 1' x 1'
patch of 64 sky positions x 2048 f1dot x 8 f2dot).  One step is one sky
position of that bank: the per-sky work (Sec. 3 steps iii-v) plus steps
vi-vii for its 16 384 spindown templates, 2F written for every bin.  Every
sky position costs the same, so templates/s of a step is the job's rate;
replicas (--gpus N) take different sky positions.

Printed JSON line: templates/s (value), 2F-bins/s, the dominant kernel's
roofline from a serialised pass (one template stream, so no other kernel
overlaps the events), the whole path's HBM and FP32 fractions against
measured peaks, the FP64-GPU comparison path, cuFFT for the same
transforms, the oracle on the host cores, end-to-end through host buffers
(e2e: pinned x_h up, 2F reduced on the device to band maxima and 2F > 70,
results down), further workloads (the 10-day narrowband search, one CUDA
graph, uneven targets, refinement, semi-coherent segments, interpolator
costs), and clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import dataclasses
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
WORKLOAD = ("large narrowband search, one sky position per step: H1+L1, 120 d, dt=1 s, "
            "10,368,000 c64 samples/det, FFT 2^24, per-sky work + 2048 f1dot x 8 f2dot = 16,384 "
            "templates (1 of the 64 sky positions of the 1'x1' patch bank), Dterms 8")
NARROW = ("narrowband single target: H1+L1, 10 d, dt=0.5 s, 1,728,000 c64 samples/det, "
          "FFT 2^22, 1 sky x 8192 f1dot x 4 f2dot = 32,768 templates, Dterms 8")


def headline_config(world: int) -> dict:
    """The ``config`` object both arms print (the driver compares them)."""
    return {"workload": WORKLOAD, "templates_per_step": 16384, "sky_positions_in_job": 64,
            "n_fft": 1 << 24, "n_samples": 10_368_000,
            "l2": "flushed between steps (256 MB write, untimed); inputs (2 x 83 MB x_h, 166 MB "
                  "resampled series) exceed the 126 MB L2",
            "parallelism": f"replicas x{world}"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=64, help="templates per fstat_compute call")
    ap.add_argument("--extra-steps", type=int, default=3, help="timed steps of the further workloads")
    ap.add_argument("--fp64-templates", type=int, default=4)
    for leg in ("e2e", "cpu", "fp64", "refine", "graph", "uneven", "narrow", "interp", "semicoh", "skyheavy",
                "sft", "cufft", "probe"):
        ap.add_argument(f"--no-{leg}", action="store_true")
    ap.add_argument("--streams", type=int, default=0, help="template streams per plan (0 = the plan's default)")
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


def ncu_traffic(kernel: str, length: int, c: int, v: int, workload: str):
    """DRAM bytes per launch of one pass shape (FFT length, columns or rows
    per CTA, radix schedule) on one workload ("large" or "narrow") from the
    committed ncu summary, if it was taken on the current kernel source
    (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        if t.get("source_hash") != kernel_source_hash():
            return None
        for e in t["entries"]:
            if (e["kernel"], e["L"], e["c"], e["v"], e.get("workload")) == (kernel, length, c, v, workload):
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
def oracle_sample(t, xs, sky, n_tmpl, warmup=0, part=8):
    """The FP64 oracle as it stands, on a bounded sample of one sky
    position's work: the per-sky step (iii-v) on the first 1/part of the
    samples (its cost is linear in the sample count, so it is scaled by
    part), then steps vi-vii of ``warmup`` untimed and ``n_tmpl`` timed
    templates at the full size (the full-length per-sky series is the
    sample's, repeated; the FFT's cost does not depend on the values).
    Returns (per-sky seconds, [per-template seconds])."""
    from oracle import resamp

    n = t.n_samples // part
    ts = dataclasses.replace(t, n_samples=n, injections=(), name=t.name + ".sample")
    s = time.perf_counter()
    prep = resamp.sky_prep(ts, [np.asarray(x[:n], dtype=np.complex128) for x in xs], *sky)
    t_sky = (time.perf_counter() - s) * t.n_samples / n
    full = dict(prep)
    full["Ga"] = np.resize(prep["Ga"], t.n_samples)
    full["Gb"] = np.resize(prep["Gb"], t.n_samples)
    f1, f2 = t.f1dots, t.f2dots
    for k in range(warmup):
        resamp.twoF(t, full, float(f1[k % len(f1)]), float(f2[0]))
    times = []
    for k in range(n_tmpl):
        s = time.perf_counter()
        resamp.twoF(t, full, float(f1[(k + warmup) % len(f1)]), float(f2[k % len(f2)]))
        times.append(time.perf_counter() - s)
    return t_sky, times


def _oracle_worker(job):
    """One host process of the all-cores oracle timing: steps vi-vii of
    ``k`` templates of the full size on seeded per-sky series."""
    t, seed, k = job
    from oracle import resamp

    rng = np.random.default_rng(seed)
    prep = {"Ga": rng.standard_normal(t.n_samples) + 1j * rng.standard_normal(t.n_samples),
            "Gb": rng.standard_normal(t.n_samples) + 1j * rng.standard_normal(t.n_samples),
            "A": 1.0, "B": 1.0, "C": 0.1, "D": 0.99, "t_b0": t.t0}
    times = []
    for i in range(k):
        s = time.perf_counter()
        resamp.twoF(t, prep, float(t.f1dots[i]), float(t.f2dots[0]))
        times.append(time.perf_counter() - s)
    return times


def cpu_oracle_all_cores(t, t_sky_1core, n_tmpl, n_per_worker=1):
    """Steps vi-vii of the oracle in one spawned process per host core, all
    at once; the per-sky step enters as its 1-core time spread over the
    cores (it splits into independent sample ranges)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    workers = os.cpu_count() or 1
    jobs = [(t, 1000 + w, n_per_worker) for w in range(workers)]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_oracle_worker, jobs))
    t_tmpl = statistics.median(x for r in res for x in r)
    value = n_tmpl / ((t_sky_1core + n_tmpl * t_tmpl) / workers)
    return {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} spawned processes at once, each {n_per_worker} template(s) of steps vi-vii "
                      f"at FFT 2^{int(math.log2(t.n_fft))} (median {t_tmpl:.2f} s); per-sky step "
                      f"{t_sky_1core:.1f} s (1 core, from a 1/8 sample) spread over the cores; "
                      f"{n_tmpl} templates per sky position"}


# ------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands on the host cores, on
    the headline workload's sky position.  Each timed step is one template
    of steps vi-vii at full size (2 x 2^24-point FFTs); the per-sky step is
    timed once on a 1/8 sample and scaled.  value = templates/s of a whole
    sky position (per-sky step + 16 384 templates)."""
    if rank != 0:
        return
    t = config5()
    xs = make_inputs(t, 0)
    t_sky, times = oracle_sample(t, xs, t.skies[0], args.steps, warmup=args.warmup)
    n = 16384
    t_tmpl = sum(times) / len(times)
    value = n / (t_sky + n * t_tmpl)
    sample = (f"per-sky step {t_sky:.1f} s (timed on 1/8 of the samples, scaled by 8) + {args.steps} timed "
              f"template(s) of steps vi-vii at {t_tmpl:.2f} s each after {args.warmup} untimed; value = "
              f"{n} / (per-sky + {n} x per-template)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_tmpl * 1e3,
            "step": "one template of steps vi-vii (the oracle's unit of work); ms_per_step is its measured time",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": headline_config(world),
            "setup": {"precision": "FP64 throughout (the oracle, NumPy complex128)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
PASS_BYTES = {0: "pass_a", 1: "pass_b", 3: "fused"}


def serial_roofline(plan, t, tm, out, stream, n=32):
    """Per-kernel CUDA-event times from a serialised pass (one template
    stream: no other kernel of the plan overlaps a launch's events), and
    each kernel's algorithmic bytes per launch: pass A reads G_a, G_b
    (16 B per sample), pass B writes 2F (4 B per bin), a fused launch does
    both for every template it covers.  Returns {kind: (launches, total ms,
    bytes per launch)}."""
    plan.set_streams(1)
    plan.compute_ptr(tm[:2], out.data_ptr(), stream)
    plan.sync()
    plan.set_profiling(True)
    plan.compute_ptr(tm[:n], out.data_ptr(), stream)
    plan.sync()
    res = {}
    for k in (0, 1, 3):
        nl, tot = plan.kernel_stats(k)
        if nl:
            per_launch = {0: 16.0 * t.n_samples, 1: 4.0 * t.n_fft,
                          3: (16.0 * t.n_samples + 4.0 * t.n_fft) * n / max(nl, 1)}[k]
            res[k] = (nl, tot, per_launch)
    plan.set_profiling(False)
    return res


def roofline_line(serial, t, value_per_gpu, hbm_peak, peak_kind, f32_peak, f32_kind, plan, ms_per_template,
                  workload):
    dom = max(serial, key=lambda k: serial[k][1])
    nl, tot, bytes_alg = serial[dom]
    avg_s = tot / 1e3 / nl
    achieved = bytes_alg / avg_s / 1e9
    n1, n2 = plan.split
    ca, va, cb, vb = plan.cta
    shape = {0: (n2, ca, va), 1: (n1, cb, vb), 3: (n1 * n2, ca, cb)}[dom]
    bpt = 16.0 * t.n_samples + 4.0 * t.n_fft
    flops_t = 2 * 5 * t.n_fft * math.log2(t.n_fft)
    serial_ms = sum(v[1] / v[0] for k, v in serial.items() if k in (0, 1))
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": ncu_traffic(PASS_BYTES[dom], *shape, workload),
            "kernel": PASS_BYTES[dom], "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, copy)",
            "timing": f"serialised pass: one template stream, {nl} launches, CUDA events per launch",
            "kernel_ms_per_launch": avg_s * 1e3, "bytes_per_launch": bytes_alg,
            "kernels": {PASS_BYTES[k]: {"launches": v[0], "ms_per_launch": v[1] / v[0],
                                        "GBps": v[2] / (v[1] / v[0] / 1e3) / 1e9,
                                        "frac": v[2] / (v[1] / v[0] / 1e3) / 1e9 / hbm_peak}
                        for k, v in serial.items()},
            "serialised_ms_per_template": serial_ms if serial_ms else None,
            "pipelined_ms_per_template": ms_per_template,
            "path": {"bytes_per_template": bpt, "achieved_GBps": bpt * value_per_gpu / 1e9,
                     "frac": bpt * value_per_gpu / 1e9 / hbm_peak},
            "alu": {"unit": "TFLOP/s", "peak": f32_peak, "peak_source": f32_kind,
                    "flops_per_template": flops_t,
                    "path_achieved": flops_t * value_per_gpu / 1e12,
                    "path_frac": flops_t * value_per_gpu / 1e12 / f32_peak},
            "split": [n1, n2], "cta": list(plan.cta)}


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

    # measured FMA peaks of this GPU (denominators of the ALU fractions)
    probe = None
    if not args.no_probe:
        f32, ms32 = pkg.probe_fma(pkg.MIXED, 1 << 16, stream)
        f64, ms64 = pkg.probe_fma(pkg.FP64, 1 << 12, stream)
        probe = {"fp32_fma_tflops": f32, "fp64_fma_tflops": f64, "fp32_ms": ms32, "fp64_ms": ms64,
                 "how": "fstat_probe_fma: 8 independent FMA chains per thread, 2048 threads per SM on every "
                        "SM, CUDA events, after one warm-up launch"}

    t = config5()
    xs = make_inputs(t, rank)
    sky = t.skies[rank % len(t.skies)]
    tm = pkg.as_templates(template_grid((sky,), t.f1dots, t.f2dots))
    n_tmpl = len(tm)
    chunk = min(args.chunk, n_tmpl)
    n_fft = t.n_fft

    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    if args.streams:
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
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = plan.launches
    for k in range(args.steps):
        flush.zero_()                      # untimed: evict L2 between steps
        barrier()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        barrier()
    launches = plan.launches - l0
    plan.sync()
    clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms = reduce_max(ms, world, dev)
    total_tmpl = n_tmpl * args.steps * world
    value = total_tmpl / (ms / 1e3)
    per_gpu = value / world
    hbm_peak, peak_kind = peaks()
    serial = serial_roofline(plan, t, tm, out, stream)
    f32_peak, f32_kind = ((probe["fp32_fma_tflops"], "measured: fstat_probe_fma FP32") if probe else
                          (torch.cuda.get_device_properties(dev).multi_processor_count * 128 * 2 * 2.07e9 / 1e12,
                           "derived: SMs x 128 FP32 lanes x 2 x 2070 MHz"))
    roof = roofline_line(serial, t, per_gpu, hbm_peak, peak_kind, f32_peak, f32_kind, plan,
                         ms / args.steps / n_tmpl, "large")
    split, cta = plan.split, plan.cta
    plan.close()
    del out

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "bins_per_s": value * n_fft,
                "tau_F_eff_s": 1.0 / (value * n_fft * len(t.detectors)),
                "job_hours_64_sky": 64 * n_tmpl / per_gpu / 3600.0,
                "config": headline_config(world),
                "setup": {"precision": "mixed: FP64 timing and phases, FP32 resample/FFT/2F",
                          "chunk": chunk, "streams": args.streams or "plan default"},
                "roofline": roof, "gpu_launches": launches, "clocks": clocks.summary()}
        if probe:
            line["peaks_probe"] = probe
        line["setup"]["shape"] = {"split": list(split), "cta": list(cta)}

    def leg(name, fn, flag=None):
        # a further workload; its failure is reported, not fatal to the line
        if rank != 0 or getattr(args, "no_" + (flag or name.split("_")[0]), False):
            return
        try:
            line[name] = fn()
        except Exception as e:  # noqa: BLE001
            line[name] = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.synchronize(dev)

    ksteps = max(1, min(args.steps, args.extra_steps))
    # FP64-GPU comparison path (same kernels in FP64) on the headline workload
    leg("fp64_gpu", lambda: fp64_gpu(t, xs, tm, args.fp64_templates, dev, stream, per_gpu))
    # cuFFT (through torch.fft) for the same transforms, comparison only
    leg("cufft", lambda: cufft_bench(dev, stream, per_gpu))
    # the radix-16 stage on CUDA cores vs as a matmul on the tensor cores
    leg("dft16_stage", lambda: dft16_stage(dev, stream), "probe")
    # end to end through the public API: pinned host x_h -> device, every
    # bin's 2F reduced on the device (band maxima and 2F > 70, the retention
    # of Sec. 5.4), results back to pinned host memory
    leg("e2e", lambda: e2e_peaks(t, xs, tm, chunk, dev, stream, args, ksteps))
    xs = None
    # the 10-day narrowband search (FFT 2^22) as before, and further workloads
    t2 = config2()
    xs2 = make_inputs(t2, rank)
    tm2 = pkg.as_templates(t2.templates())
    leg("narrow", lambda: narrow_bench(t2, xs2, tm2, dev, stream, args, ksteps, flush, hbm_peak, peak_kind,
                                       f32_peak, f32_kind))
    leg("graph", lambda: graph_bench(t2, xs2, tm2, 256, dev, stream, ksteps, flush))
    leg("uneven_targets", lambda: uneven_bench(dev, stream, ksteps))
    leg("sky_heavy", lambda: sky_heavy_bench(t2, xs2, dev, stream, ksteps), "skyheavy")
    leg("sft_to_xh", lambda: sft_bench(t2, dev))
    leg("semicoherent", lambda: semicoh_bench(dev, stream, ksteps), "semicoh")
    leg("interp_cost", lambda: interp_cost(t2, xs2, tm2, dev, stream))
    leg("refine", lambda: refine_bench(t2, xs2, dev))
    leg("e2e_dense_narrowband", lambda: e2e(t2, xs2, tm2, 256, dev, stream, 1), "e2e")

    if rank == 0 and not args.no_cpu:
        xs = make_inputs(t, 0)
        t_sky, times = oracle_sample(t, xs, sky, 2)
        t_tmpl = sum(times) / len(times)
        cpu_v = n_tmpl / (t_sky + n_tmpl * t_tmpl)
        line["cpu_baseline"] = {
            "value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"per-sky step {t_sky:.1f} s (timed on 1/8 of the 2 x 10,368,000 samples, scaled by 8) + "
                      f"2 templates of steps vi-vii (2 x 2^24-point FFTs) at {t_tmpl:.2f} s each; value = "
                      f"{n_tmpl} / (per-sky + {n_tmpl} x per-template)"}
        line["cpu_baseline_all_cores"] = cpu_oracle_all_cores(t, t_sky, n_tmpl)
    if rank == 0:
        print(json.dumps(line), flush=True)


def cufft_bench(dev, stream, mixed_value, reps=10):
    """cuFFT through torch.fft on the same transforms as one template's
    steps vi-vii (two complex64 C2C transforms of 2^24 and of 2^22 points),
    timed with CUDA events after warm-up; comparison only (the library's
    FFT is its own)."""
    import torch

    res = {}
    for log2n in (22, 24):
        x = torch.randn((2, 1 << log2n), dtype=torch.complex64, device=dev)
        for _ in range(3):
            torch.fft.fft(x)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            torch.fft.fft(x)
        b.record(stream)
        torch.cuda.synchronize(dev)
        res[f"2x2^{log2n}_ms"] = a.elapsed_time(b) / reps
        del x
    res["note"] = ("two C2C transforms only (no spindown phase, no 2F, no zero-padding skip); the library's "
                   "whole template at 2^24 takes 1/value")
    res["ours_ms_per_template_2e24"] = 1e3 / mixed_value
    return res


def dft16_stage(dev, stream, blocks=1216, reps=64):
    """The radix-16 DFT stage of the FFT passes on the CUDA cores (the
    passes' butterflies) and as a TF32 matrix product on the tensor cores
    (three-term split for FP32-level accuracy), same vectors, staged in
    shared memory and transformed `reps` times: ns per 16-point vector."""
    import torch

    import paper_2201_00451_gb300 as pkg

    n = 512 * blocks
    x = torch.randn(n * 32, dtype=torch.float32, device=dev)
    res = {}
    for method, name in ((0, "cuda_cores"), (1, "tensor_cores_3xtf32")):
        _, ms = pkg.probe_dft16(method, x, reps, stream)
        res[name + "_ns_per_vector"] = ms * 1e6 / (n * reps)
    res["tensor_over_cuda_time"] = res["tensor_cores_3xtf32_ns_per_vector"] / res["cuda_cores_ns_per_vector"]
    res["vectors"] = n
    res["reps"] = reps
    return res


def narrow_bench(t, xs, tm, dev, stream, args, steps, flush, hbm_peak, peak_kind, f32_peak, f32_kind,
                 chunk=256):
    """The 10-day narrowband search (FFT 2^22, 32 768 templates of one sky
    position per step, per-sky work included, L2 flushed between steps),
    and its serialised per-kernel roofline."""
    import torch

    import paper_2201_00451_gb300 as pkg

    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, xs[X], t.sigmas[X])
    plan.autotune(stream)
    out = torch.empty((chunk, t.n_fft), dtype=torch.float32, device=dev)
    chunks = [tm[i:i + chunk] for i in range(0, len(tm), chunk)]

    def step():
        plan.invalidate_sky()
        for c in chunks:
            plan.compute_ptr(c, out.data_ptr(), stream)

    step()
    torch.cuda.synchronize(dev)
    ms = 0.0
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms += a.elapsed_time(b)
    value = len(tm) * steps / (ms / 1e3)
    serial = serial_roofline(plan, t, tm, out, stream)
    roof = roofline_line(serial, t, value, hbm_peak, peak_kind, f32_peak, f32_kind, plan, ms / steps / len(tm),
                         "narrow")
    plan.close()
    return {"value": value, "unit": UNIT, "bins_per_s": value * t.n_fft, "ms_per_step": ms / steps,
            "workload": NARROW, "roofline": roof}


SEMI_SEGMENTS = 10


def semicoh_bench(dev, stream, steps, n_f1=256, n_f2=2):
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

    step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) * 1e-3 / steps
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
    """The plain FP64-GPU path (the same kernels in FP64, complex128 FFT) on
    the headline workload: per-sky work plus n templates, extrapolated to
    one sky position's bank."""
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
    total = len(tm_all)
    v = total / ((ms_sky + total * per_t) / 1e3)
    return {"value": v, "unit": UNIT, "sample": f"per-sky step ({ms_sky:.1f} ms) + {n} templates at "
                                               f"{per_t:.2f} ms, extrapolated to {total} templates",
            "mixed_over_fp64": mixed_value / v}


def graph_bench(t, xs, tm, chunk, dev, stream, steps, flush):
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
    batch.launch(stream)
    torch.cuda.synchronize(dev)
    ms = 0.0
    for _ in range(steps):
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
    return {"value": len(tm) * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "graph_nodes": nodes, "workload": NARROW + ", the step captured once as one CUDA graph"}


def uneven_bench(dev, stream, steps):
    """Four targets with different spans, bands and FFT lengths (2^18..2^22,
    561..13333 templates), all in one CUDA graph; seeded noise; one
    untimed replay, then ``steps`` timed replays."""
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
    batch.launch(stream)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        batch.launch(stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    nodes = batch.nodes
    batch.close()
    for p in plans:
        p.close()
    return {"value": n_tmpl / (ms / 1e3), "unit": UNIT, "bins_per_s": n_bins / (ms / 1e3),
            "targets": [{"n_samples": tg.n_samples, "n_fft": tg.n_fft, "templates": tg.n_templates,
                         "f_het": tg.f_het} for tg in targets],
            "ms_per_replay": ms, "replays": steps, "graph_nodes": nodes}


def sky_heavy_bench(t, xs, dev, stream, steps, n_sky=128, n_f1=11):
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
    plan.compute_ptr(tm, out.data_ptr(), stream)
    torch.cuda.synchronize(dev)
    plan.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.invalidate_sky()
        plan.compute_ptr(tm, out.data_ptr(), stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sec = e0.elapsed_time(e1) * 1e-3 / steps
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


def e2e(t, xs, tm, chunk, dev, stream, steps):
    """The 10-day search end to end with every bin's 2F read back (550 GB
    per step) into pinned host memory: bound by the device-to-host copy."""
    import torch

    import paper_2201_00451_gb300 as pkg

    n_fft = t.n_fft
    hx = [torch.from_numpy(x).pin_memory() for x in xs]
    plan = pkg.FstatPlan.from_target(t, pkg.MIXED)
    for X in range(len(t.detectors)):
        plan.set_data(X, hx[X].numpy(), t.sigmas[X])
    plan.autotune(stream)               # the autotuner's choice from its in-process cache
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

    step()
    torch.cuda.synchronize(dev)
    s = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - s
    plan.close()
    n = len(tm) * steps
    return {"value": n / el, "unit": UNIT, "workload": NARROW,
            "h2d_bytes_per_step": int(sum(x.nbytes for x in xs)),
            "d2h_bytes_per_step": int(len(tm) * n_fft * 4)}


PEAK_BANDS = 256         # band maxima per template (W = 65536 bins = 3.9 mHz at FFT 2^24, dt 1 s)
PEAK_THRESHOLD = 70.0    # the retention threshold of Sec. 5.4
PEAK_CAPACITY = 1 << 16


def e2e_peaks(t, xs, tm, chunk, dev, stream, args, steps):
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
    for _ in range(steps):
        step()
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - s
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(with_copies=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dev_s = e0.elapsed_time(e1) * 1e-3
    n_cross = int(hcount.sum())
    peaks_shape = list(plan.peaks_cta)
    plan.close()
    n = len(tm) * steps
    return {"value": n / el, "unit": UNIT,
            "h2d_bytes_per_step": int(sum(x.nbytes for x in xs)),
            "d2h_bytes_per_step": int(hmax.nbytes + hbin.nbytes + hcount.nbytes + hpeaks.nbytes),
            "output": f"{PEAK_BANDS} band maxima (2F, bin) per template + list of 2F > {PEAK_THRESHOLD:g}",
            "crossings_per_step": n_cross,
            "device_value": n / dev_s, "pass_b_shape": peaks_shape}


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
