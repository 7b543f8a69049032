"""Benchmark of the Bragg-spot sum on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the large shot (3072x3072 pixels, oversample 2, 2 sensor layers,
100 sources on a 0.5 % Gaussian spectrum at 9.5 keV, 50 mosaic domains,
Na=Nb=Nc=25 Gaussian shape, tricubic F_cell on hkl in [-60,60]^3, Kahn
0.99): 3.77e11 pixel-steps per image.  One step = one image: the per-shot
host set-up (rotated axes, source tables) and the whole per-pixel sum with
the fused double accumulate, in the FP32-mixed form.  The JSON line also
carries the plain FP64 form (timed on a strided pixel subset of the same
shot, its rate scaled by nothing: pixel-steps it did / time it took).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA
events on the library's stream; a 512 MB buffer is rewritten between timed
steps (outside the events) to flush the 129 MB L2.  Multi-GPU (torchrun):
independent replicas, one shot per rank, no data-path collective; the
slowest rank's time sets the rate.

The oracle leg (`cpu`, rank 0 at N=1) times the FP64 CPU oracle on a row
sample of the large shot (cpu_baseline) and reports every form's error
against it per configuration: the single shot and the precision sweep
(N = 10, 50, 200), with each form's full-image time (precision).

--impl reference times the FP64 CPU oracle (the only reference this method
has: the paper ships no code) on the host cores, on a strided row sample of
the same shot per step.
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

METRIC = ("pixel-steps/s (FP32-mixed vs FP64 form); served shots/s with "
          "p99 latency")
UNIT = "pixel-steps/s"
WORKLOAD = ("large shot 3072x3072, oversample 2, 2 layers (0.5 mm, atten "
            "0.3 mm), 100 sources (0.5% Gaussian at 9.5 keV), 50 mosaic "
            "domains, cell 79x79x38 A, N=25 Gaussian, tricubic F on "
            "[-60,60]^3, Kahn 0.99")
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0  # GB300's maximum SM clock
# DRAM bytes (read + write) of one full-size launch of the warp-per-pixel
# kernel, from one ncu capture (profiles/spots_split_large_shot_dram.txt:
# the mean of two launches);
# valid only while the kernel sources hash to the value they had then
TRAFFIC_CAPTURE = {"bytes": (80408320 + 22961920 + 80121344 + 23371520) // 2,
                   "sources": ["paper_2205_07976_gb300/csrc/spots_split.cu",
                               "paper_2205_07976_gb300/csrc/split_pixel.cuh",
                               "paper_2205_07976_gb300/csrc/mixed_common.cuh",
                               "paper_2205_07976_gb300/csrc/nbgb_internal.cuh"],
                   "sha256_16": "068389bc3a988e15"}


def captured_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_CAPTURE["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != TRAFFIC_CAPTURE["sha256_16"]:
        return None
    return TRAFFIC_CAPTURE["bytes"]


# Pipe utilisation (% of active cycles) of the warp-per-pixel kernel from
# one ncu --set full capture on a 512x512 window of the large shot
# (profiles/spots_split_window512_full.txt), keyed like the traffic figure
PIPES_CAPTURE = {"sm__pipe_fma_cycles_active_pct": 36.3,
                 "sm__pipe_alu_cycles_active_pct": 40.1,
                 "sm__inst_executed_pipe_lsu_pct": 41.3,
                 "smsp__issue_active_pct": 74.1,
                 "l1tex__data_pipe_lsu_wavefronts_pct": 54.5,
                 "window": "512x512 centred on the large shot",
                 "sha256_16": "068389bc3a988e15"}


def captured_pipes():
    """ncu's pipe utilisation of the current kernel, or None once its
    sources changed since the capture."""
    if PIPES_CAPTURE is None:
        return None
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_CAPTURE["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != PIPES_CAPTURE["sha256_16"]:
        return None
    return {k: v for k, v in PIPES_CAPTURE.items() if k != "sha256_16"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--f64-rows-every", type=int, default=96)
    ap.add_argument("--window", type=int, default=0,
                    help="time an N x N window of the large shot instead "
                         "of the whole image (for profiling)")
    ap.add_argument("--legs", default="main,e2e,f64,cpu,serve,bkg,grad",
                    help="comma list of main, e2e, f64, cpu (the oracle "
                         "leg: cpu_baseline and the per-config errors), "
                         "serve, bkg, grad")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-seq-subset", type=int, default=16)
    ap.add_argument("--serve-budget", type=int, default=2_000_000_000,
                    help="pixel-steps per serving step")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        # samples under load: the upper half of the observed clocks
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- helpers


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(shot, every: int, threads: int = 0):
    import oracle
    from paper_2205_07976_gb300 import workloads as W
    pix = W.strided_rows(shot, every)
    oracle.build()
    t0 = time.perf_counter()
    oracle.image(shot, pix, nthreads=threads)
    dt = time.perf_counter() - t0
    steps = len(pix) * shot.steps_per_pixel
    # one thread, on the first 1024 pixels of that sample
    one = pix[:1024]
    t1 = time.perf_counter()
    oracle.image(shot, one, nthreads=1)
    d1 = time.perf_counter() - t1
    return {"value": steps / dt, "unit": UNIT,
            "cores": threads or oracle.max_threads(), "kind": "oracle",
            "sample": f"every {every}th row of the large shot "
                      f"({len(pix)} pixels, {steps:.3e} pixel-steps, "
                      f"{dt:.1f} s)",
            "single_thread_value": len(one) * shot.steps_per_pixel / d1,
            "single_thread_sample": f"{len(one)} of those pixels, {d1:.1f} s"}


# ------------------------------------------------------------ our arm


def run_ours(args):
    import numpy as np
    import torch
    from paper_2205_07976_gb300 import nbgb
    from paper_2205_07976_gb300 import workloads as W

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    legs = set(args.legs.split(","))
    shot = W.large_shot(seed=1 + rank)
    if args.window:
        shot = W.shrink(shot, args.window, args.window, 1024, 1024)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32,
                        device=dev)
    sim = nbgb.Sim("mixed", device=local, stream=stream).set_shot(shot)
    sim.set_variant("warp")  # the warp-per-pixel kernel (spots_split_kernel)

    kernel_times = []

    def step(record=False):
        # per-shot host set-up (a1) + the whole per-pixel sum (a2..a8)
        sim.set_crystal(shot, with_F=False)
        if record:
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            sim.add_spots()
            k1.record(stream)
            kernel_times.append((k0, k1))
        else:
            sim.add_spots()

    def timed(fn, k):
        times = []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            fn(record=True)
            ev1.record(stream)
            stream.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
        return times

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = timed(step, args.steps)
    torch.cuda.synchronize()
    barrier(pg)
    t_step = max_over_ranks(pg, sum(times) / len(times))
    units = shot.pixel_steps * world
    value = units / t_step
    clocks = clk.summary()

    serving = None
    if "serve" in legs:
        serving = run_serving(args, local, torch, nbgb, W)
    e2e = None
    if "e2e" in legs:
        e2e = run_e2e(args, sim, shot, world, pg, torch, np, nbgb)
    f64 = None
    if "f64" in legs:
        f64 = run_f64(args, shot, local, stream, torch, nbgb, W)
    differentiation = None
    if "grad" in legs:
        differentiation = run_grad(args, local, stream, torch, nbgb, W)
    background = None
    if "bkg" in legs:
        background = run_background(args, shot, local, stream, flush, torch,
                                    nbgb, W)

    if rank != 0:
        return
    from paper_2205_07976_gb300 import flops
    evaluated, _ = sim.stats()  # terms evaluated by the last timed launch
    # one more launch, untimed, with the counting instantiation: what a
    # launch performs (the counts depend only on the inputs)
    sim.count_work(True)
    sim.zero()
    step()
    work = sim.work()
    sim.count_work(False)
    t_kernel = sum(a.elapsed_time(b) for a, b in kernel_times) / 1e3 / len(
        kernel_times)
    alg = flops.algorithmic_flops(shot, evaluated)
    performed = flops.performed_flops(shot, work)
    achieved = alg / t_kernel / 1e12
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    peak_fp32 = flops.fp32_peak_tflops(sm_count, MAX_SM_MHZ)
    sm_mhz = clocks["sm_mhz"] if clocks else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "pixels": shot.npix,
                   "steps_per_pixel": shot.steps_per_pixel,
                   "pixel_steps_per_image": shot.pixel_steps,
                   "precision": "FP32-mixed", "parallelism": "replicas",
                   "l2": "512 MB buffer rewritten between timed steps"},
        "e2e": e2e,
        "f64": f64,
        "serving": serving,
        "background": background,
        "differentiation": differentiation,
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved,
                     "peak": peak_fp32, "unit": "TFLOP/s",
                     "frac": achieved / peak_fp32,
                     "traffic": None if args.window else captured_traffic(),
                     "kernel": "spots_split_kernel",
                     "kernel_ms": t_kernel * 1e3,
                     "algorithmic_tflop_per_launch": alg / 1e12,
                     "evaluated_terms": evaluated,
                     "sm_count": sm_count,
                     "peak_source": f"{sm_count} SMs (queried) x 128 FP32 "
                                    "lanes x 2 flops x 2070 MHz (derived "
                                    "from unit counts; FP32 is not in "
                                    "MEASURED_PEAKS)",
                     "frac_at_measured_clock": (
                         achieved / flops.fp32_peak_tflops(sm_count, sm_mhz)
                         if sm_mhz else None),
                     "performed_tflop_per_launch": performed / 1e12,
                     "frac_performed": performed / t_kernel / 1e12
                     / peak_fp32,
                     "work": work,
                     "ncu_pipes": captured_pipes()},
        "clocks": clocks,
    }
    if args.window:
        line["config"]["window"] = f"{args.window}x{args.window} pixels"
    if world == 1 and not args.no_cpu_baseline and "cpu" in legs:
        line["cpu_baseline"] = cpu_baseline(shot, 192)
        # the oracle leg also gives each form's error per configuration
        line["precision"] = run_precision(args, local, stream, torch, np,
                                          nbgb, W)
    print(json.dumps(line), flush=True)


def run_e2e(args, sim, shot, world, pg, torch, np, nbgb):
    """The same metric end to end through the C ABI with host buffers: the
    shot's inputs (F table from pinned memory, crystal, beam, detector)
    copied in and the float image copied out every step."""
    img_host = torch.empty(shot.npix, dtype=torch.float32).pin_memory()
    F_host = torch.from_numpy(np.ascontiguousarray(shot.F)).pin_memory()
    s2 = shot.copy()
    s2.F = F_host.numpy()

    def step_e2e():
        sim.set_crystal(s2, with_F=True)
        sim.set_beam(s2)
        sim.set_detector(s2)
        sim.add_spots()
        nbgb._check(sim.lib.nb_get_image(sim.h, nbgb._vp(img_host.data_ptr()),
                                         shot.npix, nbgb.NB_DTYPE_F32, 0),
                    sim.h)

    step_e2e()
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    barrier(pg)
    t_e2e = max_over_ranks(pg, (time.perf_counter() - t0) / args.steps)
    h2d = (shot.F.nbytes + shot.umats.nbytes + shot.axes.nbytes
           + shot.dirs.nbytes + shot.lambdas.nbytes + shot.weights.nbytes)
    return {"value": shot.pixel_steps * world / t_e2e, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(shot.npix * 4),
            "ms_per_step": t_e2e * 1e3}


def run_f64(args, shot, local, stream, torch, nbgb, W):
    """The plain FP64 form on every n-th row of the same shot."""
    rows = W.strided_rows(shot, args.f64_rows_every)
    sim64 = nbgb.Sim("f64", device=local, stream=stream).set_shot(shot)
    sim64.add_spots(rows)
    stream.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim64.add_spots(rows)
    ev1.record(stream)
    stream.synchronize()
    t64 = ev0.elapsed_time(ev1) / 1e3
    sim64.close()
    from paper_2205_07976_gb300 import flops
    # roofline against the FP64 FMA rate measured on this device (the
    # kernel issues scalar FP64 FMAs; there is no FP64 figure in the
    # measured-peaks file)
    peak = nbgb.fp64_peak_tflops(local)
    achieved = flops.f64_flops(shot, len(rows)) / t64 / 1e12
    return {"value": len(rows) * shot.steps_per_pixel / t64, "unit": UNIT,
            "sample": f"every {args.f64_rows_every}th row "
                      f"({len(rows)} pixels)", "ms": t64 * 1e3,
            "roofline": {"bound": "fp64", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if peak > 0 else None,
                         "kernel": "spots_f64_kernel",
                         "peak_source": "measured: independent FP64 FMA "
                                        "chains on every SM "
                                        "(nb_fp64_peak_tflops)"}}


def run_precision(args, local, stream, torch, np, nbgb, W):
    """Error of every form against the FP64 oracle, per configuration: the
    single shot (256^2, N=10 sinc, every pixel) and the precision sweep
    (1024^2, 100 sources, 20 domains, N in {10, 50, 200} sinc; the GPU
    computes the whole image, the oracle every 16th row of it).  Relative
    error per pixel on the sampled pixels above 1e-3 of their maximum (the
    NB_MIXED gate) and, for NB_F64, above 1e-6 of it (the NB_F64 gate);
    times are CUDA events around one full-image launch (median of 3, after
    one untimed launch).  At N=200 the oracle's literal sin(pi N h)/sin(pi h)
    is compared with its reduced form on the same pixels: that difference
    is the rounding the FP64 gate has to allow at large N."""
    import oracle
    every = 16
    out = {"sample": f"oracle on every {every}th row of the 1024^2 sweep "
                     "(64 rows, 65536 pixels); every pixel of the 256^2 "
                     "shot",
           "configs": {}}

    def rel(got, ref, floor, absolute=False):
        m = ref > (floor if absolute else floor * ref.max())
        r = np.abs(got[m] - ref[m]) / ref[m]
        return float(r.max()), float(np.median(r)), int(m.sum())

    def time_form(shot, prec):
        sim = nbgb.Sim(prec, device=local, stream=stream).set_shot(shot)
        sim.add_spots()
        stream.synchronize()
        ts = []
        for _ in range(3):
            sim.zero()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sim.add_spots()
            ev1.record(stream)
            stream.synchronize()
            ts.append(ev0.elapsed_time(ev1) / 1e3)
        img = sim.image()
        sim.close()
        return float(np.median(ts)), img

    cases = [("single shot 256x256, N=10 sinc", W.single_shot_small(), None)]
    for N in (10, 50, 200):
        s = W.precision_shot(N)
        cases.append((f"precision 1024x1024, N={N} sinc", s,
                      W.strided_rows(s, every)))
    for name, shot, pix in cases:
        t0 = time.perf_counter()
        ref = oracle.image(shot, pixels=pix)
        t_orc = time.perf_counter() - t0
        npx = shot.npix if pix is None else len(pix)
        row = {"oracle_pixel_steps_per_s":
               npx * shot.steps_per_pixel / t_orc}
        for prec in ("f64", "mixed", "f32"):
            t, img = time_form(shot, prec)
            got = img if pix is None else img[pix]
            e3 = rel(got, ref, 1e-3)
            row[prec] = {"ms": t * 1e3,
                         "pixel_steps_per_s": shot.pixel_steps / t,
                         "max_rel": e3[0], "median_rel": e3[1],
                         "pixels": e3[2]}
            if prec == "f64":
                row[prec]["max_rel_above_1e-6"] = rel(got, ref, 1e-6)[0]
                # every pixel above 1e-250 photons (the FP64 gate)
                row[prec]["max_rel_above_1e-250"] = rel(got, ref, 1e-250,
                                                        True)[0]
        if shot.ncells[0] == 200:
            lit = oracle.image(shot, pixels=pix, sinc_mode="literal")
            row["oracle_literal_vs_reduced_max_rel_above_1e-6"] = rel(
                lit, ref, 1e-6)[0]
            row["oracle_literal_vs_reduced_max_rel_above_1e-250"] = rel(
                lit, ref, 1e-250, True)[0]
        out["configs"][name] = row
    return out


def run_grad(args, local, stream, torch, nbgb, W):
    """One refinement step of the differentiation workload (64 panels of
    185x194, 8 sources, 10 mosaic domains, N=15 Gaussian, nearest lookup on
    [-40,40]^3): forward image, Poisson loss with dL/dI, and the adjoint
    with the gradients of the 10 crystal parameters and of every structure
    factor.  The target is a seeded Poisson draw of the forward image."""
    import numpy as np
    U = W.random_orientation(np.random.default_rng(3))
    cell, rot = np.array([79.0, 79.0, 38.0]), np.zeros(3)
    N = np.array([15.0, 15.0, 15.0])
    dev = torch.device("cuda", local)

    def timed_step(shot):
        sim = nbgb.Sim("mixed", device=local, stream=stream).set_shot(shot)
        sim.set_params(U, cell, rot, N, 1.0)
        sim.add_spots()
        y = np.random.default_rng(7).poisson(sim.image() + 1.0)
        yd = torch.from_numpy(y.astype(np.float64)).to(dev)
        dL = torch.empty_like(yd)
        gF = torch.zeros(shot.F.size, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        for _ in range(max(args.warmup, 1)):
            sim.zero()
            sim.add_spots()
            sim.poisson_loss(yd.data_ptr(), 1.0, dL.data_ptr())
            sim.adjoint(dL.data_ptr(), gF.data_ptr())
        reps = max(args.steps, 1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        tf = tl = ta = 0.0
        for _ in range(reps):
            ev[0].record(stream)
            sim.zero()
            sim.add_spots()
            ev[1].record(stream)
            sim.poisson_loss(yd.data_ptr(), 1.0, dL.data_ptr())
            ev[2].record(stream)
            sim.adjoint(dL.data_ptr(), gF.data_ptr())
            ev[3].record(stream)
            stream.synchronize()
            tf += ev[0].elapsed_time(ev[1]) / 1e3
            tl += ev[1].elapsed_time(ev[2]) / 1e3
            ta += ev[2].elapsed_time(ev[3]) / 1e3
        sim.close()
        return tf / reps, tl / reps, ta / reps

    shot = W.multipanel_shot(8)
    tf, tl, ta = timed_step(shot)
    steps = shot.pixel_steps
    tri = shot.copy()
    tri.interp = W.INTERP_TRICUBIC
    tf3, tl3, ta3 = timed_step(tri)
    return {"workload": "64 panels of 185x194, S=8, M=10, N=15 Gaussian, "
                        "nearest F on [-40,40]^3",
            "pixel_steps_per_pass": steps,
            "forward_ms": tf * 1e3, "loss_ms": tl * 1e3,
            "adjoint_ms": ta * 1e3, "step_ms": (tf + tl + ta) * 1e3,
            "adjoint_pixel_steps_per_s": steps / ta,
            "tricubic": {"forward_ms": tf3 * 1e3, "adjoint_ms": ta3 * 1e3,
                         "step_ms": (tf3 + tl3 + ta3) * 1e3,
                         "adjoint_pixel_steps_per_s": steps / ta3},
            "unit": "pixel-steps/s"}


def run_background(args, shot, local, stream, flush, torch, nbgb, W):
    """The amorphous-background kernel over the same detector, sources,
    oversampling and layers (64-knot water-like table), both forms."""
    import numpy as np
    bg = W.amorphous_background(64)
    units = shot.npix * shot.oversample ** 2 * shot.n_layers * shot.n_src
    out = {"unit": "background pixel-steps/s",
           "pixel_steps_per_image": units,
           "table": "64 knots on [0, 1]/A"}
    for prec, reps in (("mixed", max(args.steps, 1)), ("f64", 1)):
        sim = nbgb.Sim(prec, device=local, stream=stream).set_shot(shot)
        sim.set_background(bg)
        sim.add_background()
        stream.synchronize()
        times = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sim.add_background()
            ev1.record(stream)
            stream.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
        sim.close()
        t = sum(times) / len(times)
        key = "value" if prec == "mixed" else "f64_value"
        out[key] = units / t
        out["ms" if prec == "mixed" else "f64_ms"] = t * 1e3
        if prec == "mixed":
            from paper_2205_07976_gb300 import flops
            ndir = len({tuple(d) for d in np.asarray(shot.dirs)})
            alg = flops.background_flops(shot, ndir)
            peak = flops.fp32_peak_tflops(
                torch.cuda.get_device_properties(local).multi_processor_count,
                MAX_SM_MHZ)
            out["roofline"] = {"bound": "alu", "achieved": alg / t / 1e12,
                               "peak": peak, "unit": "TFLOP/s",
                               "frac": alg / t / 1e12 / peak,
                               "kernel": "background_mixed_kernel",
                               "algorithmic_tflop_per_launch": alg / 1e12}
    return out


def run_serving(args, local, torch, nbgb, W):
    """Continuous batching of shot requests (random orientation, 1-100
    sources, 1-50 mosaic domains, ROI of 1e3-4e6 pixels, log-uniform) with
    the 3072x3072 detector and the tricubic F table resident: capacity with
    all requests queued at t=0, then Poisson arrivals at 0.5, 0.8 and 1.0 x
    that capacity (latency = arrival to image fetched to host); and, on a
    fixed subset, the same requests as sequential stand-alone launches in
    FP64 and in FP32-mixed."""
    import numpy as np
    base = W.serving_detector_shot()
    reqs = W.serving_requests(args.serve_requests, seed=5)
    total_steps = sum(r.pixel_steps for r in reqs)
    buf = np.empty(max(r.npix for r in reqs), dtype=np.float64)

    def serve(arrivals):
        srv = nbgb.Server(base, max_slots=256, pool_bytes=4 << 30,
                          step_budget=args.serve_budget, device=local)
        t0 = time.perf_counter()
        arr = {}
        lat = []
        i = 0
        n = len(reqs)
        while len(lat) < n:
            now = time.perf_counter() - t0
            while i < n and arrivals[i] <= now:
                r = reqs[i]
                rid = srv.submit(r.axes, r.umats, r.lambdas, r.weights,
                                 r.scale, r.roi)
                arr[rid] = (arrivals[i], r.npix)
                i += 1
            if not arr:
                # nothing queued or running: wait for the next arrival
                time.sleep(min(max(arrivals[i] - now, 0.0), 5e-4))
                continue
            srv.step()
            for rid in srv.completed():
                a, npx = arr.pop(rid)
                srv.result(rid, out=buf[:npx])
                lat.append(time.perf_counter() - t0 - a)
        wall = time.perf_counter() - t0
        srv.close()
        lat = np.array(lat)
        return {"shots_per_s": n / wall, "wall_s": wall,
                "pixel_steps_per_s": total_steps / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3)}

    cap = serve(np.zeros(len(reqs)))
    out = {"requests": len(reqs), "pixel_steps": total_steps,
           "step_budget": args.serve_budget, "capacity": cap, "rates": {}}
    for f in (0.5, 0.8, 1.0):
        arrivals = W.poisson_arrivals(len(reqs), f * cap["shots_per_s"],
                                      seed=int(f * 10))
        out["rates"][str(f)] = serve(arrivals)
    # sequential stand-alone launches on a fixed subset
    sub = reqs[:args.serve_seq_subset]
    for prec in ("f64", "mixed"):
        t0 = time.perf_counter()
        for r in sub:
            sim = nbgb.Sim(prec, device=local).set_shot(
                W.request_shot(base, r))
            sim.add_spots()
            sim.image()
            sim.close()
        dt = time.perf_counter() - t0
        out[f"sequential_{prec}"] = {
            "shots_per_s": len(sub) / dt,
            "pixel_steps_per_s": sum(r.pixel_steps for r in sub) / dt,
            "subset": f"first {len(sub)} requests"}
    return out


# ------------------------------------------------------- reference arm


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2205_07976_gb300 import workloads as W
    shot = W.large_shot(seed=1)
    oracle.build()
    every = 384
    pix = W.strided_rows(shot, every)
    for _ in range(args.warmup):
        oracle.image(shot, pix[:3072])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.image(shot, pix)
    dt = (time.perf_counter() - t0) / args.steps
    rate = len(pix) * shot.steps_per_pixel / dt
    cores = oracle.max_threads()
    sample = (f"every {every}th row of the large shot per step "
              f"({len(pix)} pixels, {len(pix) * shot.steps_per_pixel:.3e} "
              f"pixel-steps)")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "precision": "FP64 CPU oracle"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
