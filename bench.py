#!/usr/bin/env python
"""Benchmark: unknowns/s to residual 1e-6 of the GB300 multigrid segmentation solver.

One step = one pass of the whole method on the 1024x1024 synthetic ellipse image (FP32, 9 grids,
V(2,2), Hybrid Smoother 2): set-up from the image and markers (blur, edge detector, distance
function, their restrictions, initial level set, c1/c2), one pseudo-time step solved by FAS
V-cycles until ||L(phi)|| / ||L(phi^n)|| <= 1e-6 (norms accumulated in FP64), the end-of-step
c1/c2 update and the mask.  value = n*m / seconds per step, summed over ranks (weak scaling:
every rank solves its own image).  The L2 (129 MB) is flushed by writing 512 MB between timed
steps, since the 1024^2 working set (~55 MB) would otherwise stay resident.

--impl reference times the FP64 C oracle (the plain CPU restatement of the paper used by the
tests) on the host cores on a bounded sample of the same workload.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "unknowns/sec to residual 1e-6 (FP64 check) and smoother HBM GB/s vs peak, 1 GB300"
UNIT = "unknowns/s"
WORKLOAD = "ellipse1024"
TOL = 1e-6
MAX_CYCLES = 60


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons while running (a reader thread stamps
    each sample with the host time, so summary() can keep the samples after mark())."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.rows = []
        self.t_mark = None

    def __enter__(self):
        import threading
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        if self.p:
            def read():
                for line in self.p.stdout:
                    self.rows.append((time.time(), line))
            self.th = threading.Thread(target=read, daemon=True)
            self.th.start()
        return self

    def mark(self):
        """Samples from here on only (the sampler keeps running)."""
        self.t_mark = time.time()

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
                self.th.join(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = [r.split(",") for t, r in self.rows
                if r.count(",") >= 8 and (self.t_mark is None or t >= self.t_mark)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank, lrank = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(lrank)
    dist.init_process_group(backend)
    return rank, ws, lrank, dist


def host_info():
    """The host the CPU baseline runs on: logical cores, CPU model and RAM."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            model = None
    ram = None
    try:
        with open("/proc/meminfo") as f:
            ram = round(int(f.readline().split()[1]) / 1024 ** 2, 1)
    except Exception:
        pass
    return {"logical_cores": os.cpu_count(), "cpu_model": model, "ram_gib": ram}


def oracle_sample(img, mk, cycles_needed=None, full=False, sample_cycles=2, openmp=False):
    """Times the oracle on the workload: set-up, begin_step and `sample_cycles` V-cycles (all
    V-cycles to rho <= 1e-6 when `full`).  openmp: the all-core build of the oracle (its
    independent loops on every host core; bitwise the serial results).  Returns a dict."""
    import oracle as O
    n, m = img.shape
    p = O.params(n, m, levels=9)
    t0 = time.perf_counter()
    s = O.Solver(img.astype(np.float64), mk, p, openmp=openmp)
    t1 = time.perf_counter()
    s.begin_step()
    t2 = time.perf_counter()
    ts, hist = [], []
    limit = MAX_CYCLES if full else sample_cycles
    for _ in range(limit):
        a = time.perf_counter()
        hist.append(s.vcycle())
        ts.append(time.perf_counter() - a)
        if hist[-1] <= TOL:
            break
    s.close()
    return dict(setup=t1 - t0, begin=t2 - t1, cycle=float(np.mean(ts)), cycles_run=len(hist),
                rho=hist[-1], converged=hist[-1] <= TOL)


def run_reference(args):
    """The oracle arm: the FP64 C oracle (its all-core OpenMP build, the parallel ordering of the
    smoother) on the host cores.  Each step is the whole step of the bench workload (set-up,
    V-cycles until rho <= 1e-6, end of step), unless --sample-cycles N > 0 asks for a sample of
    N V-cycles scaled to the V-cycles the first warm-up step needed."""
    rank, ws, _, dist = dist_init()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    from paper_1807_02137_gb300 import synth
    W = synth.workload(WORKLOAD)
    img, mk = W.image, W.markers
    n, m = img.shape
    full = args.sample_cycles <= 0
    cycles_needed = None
    for w in range(args.warmup):
        r = oracle_sample(img, mk, full=(w == 0 or full), openmp=True)
        if w == 0:
            cycles_needed = r["cycles_run"]
    if cycles_needed is None:
        cycles_needed = 13
    per_step, measured = [], []
    for _ in range(args.steps):
        if full:
            r = oracle_sample(img, mk, full=True, openmp=True)
            t = r["setup"] + r["begin"] + r["cycles_run"] * r["cycle"]
            per_step.append(t)
            measured.append(t)
        else:
            r = oracle_sample(img, mk, sample_cycles=args.sample_cycles, openmp=True)
            per_step.append(r["setup"] + r["begin"] + cycles_needed * r["cycle"])
            measured.append(r["setup"] + r["begin"] + args.sample_cycles * r["cycle"])
    sec = float(np.mean(per_step))
    value = n * m / sec
    hi = host_info()
    if full:
        sample = (f"FP64 C oracle (all-core OpenMP build, {hi['logical_cores']} threads): the whole step of the "
                  f"{n}x{m} workload per timed step (set-up, {cycles_needed} V-cycles to rho <= 1e-6)")
    else:
        sample = (f"FP64 C oracle (all-core OpenMP build): set-up + begin_step + {args.sample_cycles} V-cycles per "
                  f"step, extrapolated to the {cycles_needed} V-cycles the oracle needs (first warm-up step)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{WORKLOAD}: {n}x{m} FP32 image, 12 ellipses, 8 markers, 9 grids, "
                                   f"V(2,2), tau 1, one pseudo-time step to rho <= 1e-6",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": hi["logical_cores"], "kind": "oracle",
                             "sample": sample, "extrapolated": not full, "host": hi,
                             "measured_s_per_step": float(np.mean(measured))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_ours(args):
    rank, ws, lrank, dist = dist_init()
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    W = synth.workload(WORKLOAD)
    img_np, mk = W.image.astype(np.float32), W.markers
    n, m = img_np.shape

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:   # before any GPU call: the whole step on all host cores, and 2 V-cycles on one core
            cpu = {"all": oracle_sample(img_np, mk, full=True, openmp=True),
                   "one": oracle_sample(img_np, mk, sample_cycles=2)}
        except Exception as e:  # the baseline is a report, never a reason to fail the bench
            cpu = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle", "sample": f"failed: {e}"}

    buildlib.build()
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    p = segmg.default_params(n, m)
    img = torch.as_tensor(img_np, device=dev)
    s = segmg.Solver(img, mk, p)
    st = torch.cuda.ExternalStream(s.stream_ptr, device=dev)
    mask = torch.empty((n, m), dtype=torch.uint8, device=dev)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)   # 512 MB > L2

    # fused-sweep tile shapes and the first grid of the bottom kernel: measured once before timing
    # (mg_autotune; they never change results, only speed)
    s.begin_step()
    shapes = s.autotune(reps=3)
    bottom_level, cluster_level = s.stats()["bottom_level"], s.stats()["cluster_level"]
    s.end_step()

    def step():
        s.reset(img, mk)
        c, r = s.solve_step(TOL, MAX_CYCLES)
        s.mask(out=mask)
        return c, r

    # the clock sampler starts before the warm-up: its start-up (NVML) is outside the timed steps
    clk = Clocks(lrank).__enter__()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, cycles, rhos = [], [], []
    l0 = s.stats()["launches"]
    clk.mark()
    try:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            with torch.cuda.stream(st):
                flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            c, r = step()
            b.record(st)
            b.synchronize()
            times.append(a.elapsed_time(b))
            cycles.append(c)
            rhos.append(r)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    finally:
        clk.__exit__(None, None, None)
    launches = s.stats()["launches"] - l0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = float(np.mean(times))
    ms_max = ms
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = ws * n * m / (ms_max * 1e-3)

    # end to end through the host-buffer entry point (copies inside the timed region), from and
    # to page-locked host buffers allocated once; the first call builds the context that
    # mg_segment_host keeps for the following calls of the same size, and it and the next
    # warm-up calls are untimed
    e2e_ms = []
    img_host = torch.from_numpy(np.ascontiguousarray(img_np, dtype=np.float32)).pin_memory().numpy()
    mask_host = torch.empty((n, m), dtype=torch.uint8).pin_memory().numpy()
    n_warm = max(1, args.warmup)   # the first call builds the context; warm-up calls untimed
    for k in range(0 if args.no_e2e else max(1, min(args.steps, 10)) + n_warm):
        t0 = time.perf_counter()
        segmg.segment_host(img_host, mk, p, TOL, MAX_CYCLES, 0.0, 1, mask_out=mask_host)
        if k >= n_warm:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms_max = float(np.mean(e2e_ms)) if e2e_ms else float("nan")
    if dist:
        t = torch.tensor([e2e_ms_max], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms_max = float(t.item())

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel: the fused smoother sweep on the finest grid
    hbm, peak_kind = peaks()
    s.reset(img, mk)
    s.begin_step()
    kt = s.time_kernels(0, reps=5)
    sweep_ms_eager = float(np.mean(kt[1:5]))
    # the step replays the sweeps from a graph: their mean duration there (graph boundaries
    # included) is the kernel's launch duration inside the timed steps
    sweep_ms = s.time_sweeps_graph(0, reps=8)
    bytes_per_cell = 16.125        # u, G, f (4 B each) + member masks (1/8 B) read, u (4 B) written
    achieved = bytes_per_cell * n * m / (sweep_ms * 1e-3) / 1e9
    # DRAM bytes of one finest-grid sweep launch from an ncu capture of this kernel on this grid
    # (profiles/k_sweep_tma_traffic_ellipse1024.txt): u, G, f read once, u written to L2
    traffic = 12.76e6
    roof = {"bound": "hbm", "kernel": "k_sweep_tma (TMA-staged fused Hybrid Smoother 2 sweep, finest grid)",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "peak_kind": peak_kind + " (hbm_gbs, burst copy)",
            "bytes_per_cell": bytes_per_cell, "ms_per_launch": sweep_ms,
            "ms_per_launch_eager": sweep_ms_eager,
            "timing": "mean of 32 sweeps replayed from one CUDA graph as the step runs them "
                      "(mg_time_sweeps_graph); ms_per_launch_eager: eager launches between events",
            "note": "1024^2 working set is L2-resident inside a step; see roofline_hbm for 8192^2"}
    roof_big = None
    if not args.no_hbm_roofline:
        try:
            img8, mk8, _ = synth.ellipses(8192, 8192, 96, (160, 1600), 8, 0.05, 1)
            p8 = segmg.default_params(8192, 8192)
            s8 = segmg.Solver(torch.as_tensor(img8, device=dev), mk8, p8)
            s8.begin_step()
            shapes8 = s8.autotune(reps=1)
            kt8 = s8.time_kernels(0, reps=3)
            kr8 = s8.time_residuals(0, reps=3)
            sw8 = float(np.mean(kt8[1:5]))
            ach8 = bytes_per_cell * 8192 * 8192 / (sw8 * 1e-3) / 1e9
            snap_bytes = 24.25       # pn, u, w, F read; G, f and member masks (1/4 B) written
            res_bytes = 20           # pn, u, w, F read, r written (no rhs on the finest grid)
            norm_bytes = 16          # pn, u, w, F read (per-tile partials only)
            rr_bytes = 19            # pn, u, w, F read; coarse rhs, u, u0 written (a quarter each)
            big = 8192 ** 2
            roof_big = {"bound": "hbm", "grid": "8192x8192 FP32", "unit": "GB/s", "peak": hbm,
                        "tile_shape": shapes8[0],
                        "sweep": {"ms": sw8, "achieved": ach8, "frac": ach8 / hbm, "bytes_per_cell": bytes_per_cell},
                        "snapshot": {"ms": kt8[0], "bytes_per_cell": snap_bytes},
                        "residual": {"ms": kt8[5], "bytes_per_cell": res_bytes,
                                     "note": "r written; the V-cycle runs the two kernels below instead"},
                        "residual_norm": {"ms": kr8[0], "bytes_per_cell": norm_bytes,
                                          "note": "tile kernel and final FP64 sum"},
                        "residual_restrict": {"ms": kr8[1], "bytes_per_cell": rr_bytes}}
            for k in ("snapshot", "residual", "residual_norm", "residual_restrict"):
                e = roof_big[k]
                e["achieved"] = e["bytes_per_cell"] * big / (e["ms"] * 1e-3) / 1e9
                e["frac"] = e["achieved"] / hbm
            s8.close()
        except Exception as e:
            roof_big = {"error": str(e)}

    cpu_line = None
    if cpu and "all" in cpu:
        a, o1 = cpu["all"], cpu["one"]
        hi = host_info()
        sec = a["setup"] + a["begin"] + a["cycles_run"] * a["cycle"]
        sec1 = o1["setup"] + o1["begin"] + a["cycles_run"] * o1["cycle"]
        cpu_line = {"value": n * m / sec, "unit": UNIT, "cores": hi["logical_cores"], "kind": "oracle",
                    "sample": (f"FP64 C oracle, all-core OpenMP build ({hi['logical_cores']} threads): the whole step "
                               f"of the same {n}x{m} workload ({a['cycles_run']} V-cycles to rho <= 1e-6, "
                               f"{sec:.1f} s), measured, not extrapolated"),
                    "host": hi,
                    "one_core": {"value": n * m / sec1, "cores": 1,
                                 "sample": (f"serial build: set-up + begin_step + 2 V-cycles "
                                            f"({o1['setup'] + o1['begin'] + 2 * o1['cycle']:.1f} s), extrapolated "
                                            f"to the {a['cycles_run']} V-cycles of the step")}}
    elif cpu:
        cpu_line = cpu

    # the other configurations, measured in the same run (extra keys of this line): 25000^2 mixed
    # precision with its error against the oracle on a 2048^2 crop, the 64-image batch, and the
    # learned relaxation weights (trained on recorded states, then one step at 4096^2 plain and
    # learned)
    extra = {}
    if not args.no_extra:
        for key, fn in (("config3_mixed_25000", lambda: config3_report(25000, 1, 2048, lrank)),
                        ("config4_batch_64", lambda: config4_report(64, 1, lrank)),
                        ("config5_learned_4096", lambda: learned_report([4096], "hf", 1000, 4, lrank))):
            try:
                t0 = time.perf_counter()
                extra[key] = fn()
                extra[key]["wall_s"] = time.perf_counter() - t0
            except Exception as e:   # a report, never a reason to lose the headline line
                extra[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    h2d = n * m * 4 + mk.size * 8
    d2h = n * m
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {n}x{m} FP32 image, 12 ellipses, 8 markers, 9 grids, "
                                   "V(2,2), tau 1, Spencer-Chen, one pseudo-time step to rho <= 1e-6",
                       "l2": "flushed (512 MB write) between timed steps",
                       "tile_shapes": shapes, "bottom_kernel_from_grid": bottom_level,
                       "cluster_bottom_from_grid": cluster_level,
                       "cycles_per_step": float(np.mean(cycles)), "rho_last": float(max(rhos)),
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": ws * n * m / (e2e_ms_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max, "calls_timed": len(e2e_ms),
                    "ms_min": float(np.min(e2e_ms)) if e2e_ms else None,
                    "path": "mg_segment_host (page-locked host image in, host mask out; image set-up "
                            "included, handle kept across calls of the same size)"},
            "gpu_launches": int(launches),
            "roofline": roof, "roofline_hbm": roof_big,
            "cpu_baseline": cpu_line,
            "clocks": clk.summary(),
            "wall_s_timed_region": t_wall, **extra}
    print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


def run_profile_case(args):
    """Small profiling case for ncu: an N x N ellipse image (N = --profile), one pseudo-time step
    started and `--cycles` V-cycles run with eager launches (no graph), nothing timed."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    buildlib.build()
    N = args.profile
    img, mk, _ = synth.ellipses(N, N, max(12, 12 * N // 1024), (20 * N / 1024, 200 * N / 1024), 8,
                                0.05, 1)
    p = segmg.default_params(N, N, use_graph=0)
    s = segmg.Solver(torch.as_tensor(img, device="cuda"), mk, p)
    if args.tile_shape >= 0:
        s.set_tile_shapes([args.tile_shape] * (p.levels - 1))
    s.begin_step()
    if args.autotune:        # the bench's kernel choices (tile shapes, bottom of the V-cycle)
        s.autotune(reps=3)
        s.end_step()
        s.reset(torch.as_tensor(img, device="cuda"), mk)
        s.begin_step()
    if args.shapes:          # or given explicitly (as a bench line reports them)
        s.set_tile_shapes([int(x) for x in args.shapes.split(",")])
    if args.cluster_level is not None:
        s.set_cluster_level(args.cluster_level)
    if args.time_kernels:    # the finest grid's kernels as mg_time_kernels / mg_time_residuals run them
        s.time_kernels(0, reps=1)
        s.time_residuals(0, reps=1)
    for _ in range(args.cycles):
        r = s.vcycle()
    print(json.dumps({"profile_case": N, "cycles": args.cycles, "rho": r, **s.stats()}), flush=True)
    s.close()


def run_config3(args):
    print(json.dumps(config3_report(args.config3, args.steps)), flush=True)


def config3_report(N, steps, crop_size=2048, dev_index=0):
    """Mixed precision at large size (w stored in BF16, smoothing FP32, FP64 norms and coarsest
    solve): one pseudo-time step to rho <= 1e-6 on an N x N image from the ellipse recipe
    (200 ellipses, axes 100-3000 px, 20 markers), the smoother roofline at that size, and the
    error against the FP64 oracle (its all-core build) on a crop_size^2 crop solved as a
    standalone problem.  Returns a dict."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    import oracle as O
    buildlib.build()
    dev = torch.device("cuda", dev_index)
    t0 = time.perf_counter()
    img, mk = synth.ellipses_device(N, N, 200, (100 * N / 25000, 3000 * N / 25000), 20, 0.05, 2, dev)
    gen_s = time.perf_counter() - t0
    p = segmg.default_params(N, N, precision=segmg.MG_MIXED)
    s = segmg.Solver(img, mk, p)
    st = torch.cuda.ExternalStream(s.stream_ptr, device=dev)
    s.solve_step(TOL, MAX_CYCLES)                 # warm-up (graph capture)
    times, cyc = [], []
    with Clocks(dev_index) as clk:
        for _ in range(max(1, steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            s.reset(img, mk)
            c, r = s.solve_step(TOL, MAX_CYCLES)
            b.record(st)
            b.synchronize()
            times.append(a.elapsed_time(b))
            cyc.append(c)
    hbm, _ = peaks()
    s.reset(img, mk)
    s.begin_step()
    kt = s.time_kernels(0, reps=2)
    sw = float(np.mean(kt[1:5]))
    stats = s.stats()
    s.close()
    # accuracy on a crop around the markers, solved standalone by the GPU (mixed and FP32) and
    # by the FP64 oracle
    C = min(crop_size, N)
    cx, cy = float(np.mean(mk[:, 0])), float(np.mean(mk[:, 1]))
    j0 = int(min(max(cx - C / 2, 0), N - C)); i0 = int(min(max(cy - C / 2, 0), N - C))
    crop = img[i0:i0 + C, j0:j0 + C].float().cpu().numpy().copy()
    cmk = mk - np.array([j0, i0])
    cmk = cmk[(cmk[:, 0] >= 0) & (cmk[:, 0] <= C - 1) & (cmk[:, 1] >= 0) & (cmk[:, 1] <= C - 1)]
    del img
    torch.cuda.empty_cache()
    out, taus = {}, {}
    for name, prec in (("mixed", segmg.MG_MIXED), ("f32", segmg.MG_F32)):
        pc = segmg.default_params(C, C, precision=prec)
        sc = segmg.Solver(torch.as_tensor(crop, device=dev), cmk, pc)
        sc.solve_step(TOL, MAX_CYCLES)
        out[name] = sc.phi().double().cpu().numpy()
        taus[name] = sc.stats()["tau"]
        sc.close()
    # the oracle solves the same step with the tau each GPU solve's step control accepted
    refs, hist = {}, None
    t1 = time.perf_counter()
    for tau in sorted(set(taus.values())):
        po = O.params(C, C, levels=segmg.default_params(C, C).levels, tau=tau)
        so = O.Solver(crop.astype(np.float64), cmk, po, openmp=True)
        hist = so.solve_step(1e-9, 80)
        refs[tau] = so.phi
        so.close()
    oracle_s = time.perf_counter() - t1
    acc = {}
    for name, phi in out.items():
        ref = refs[taus[name]]
        acc[name] = {"max_rel_err_phi": float(np.max(np.abs(phi - ref)) / np.max(np.abs(ref))),
                     "mask_mismatch_frac": float(np.mean((phi > 0) != (ref > 0)))}
    bytes_sweep = 16.125 * N * N
    return {"config": f"{N}x{N} mixed precision (w BF16, smoothing FP32, FP64 norms/coarsest)",
            "levels": stats["levels"], "unknowns_per_s": N * N / (np.mean(times) * 1e-3),
            "ms_per_step": float(np.mean(times)), "cycles_per_step": float(np.mean(cyc)),
            "tau": stats["tau"], "rho": float(r),
            "device_bytes": stats["device_bytes"], "generate_s": gen_s,
            "roofline_sweep": {"ms": sw, "achieved_GBs": bytes_sweep / (sw * 1e-3) / 1e9, "peak": hbm,
                               "frac": bytes_sweep / (sw * 1e-3) / 1e9 / hbm},
            "kernel_ms": {"snapshot": kt[0], "sweeps": kt[1:5], "residual": kt[5]},
            "crop": {"size": C, "origin": [i0, j0], "markers": int(len(cmk)), "tau": taus,
                     "oracle_cycles": len(hist), "oracle_rho": hist[-1], "oracle_s": oracle_s,
                     "oracle_build": "all-core OpenMP (bitwise the serial checker)", **acc},
            "clocks": clk.summary()}


def run_config4(args):
    print(json.dumps(config4_report(args.config4, args.steps)), flush=True)


def config4_report(count, steps, dev_index=0):
    """Batched uneven sizes: `count` images with sizes drawn from {256, 512, 768, 1024, 2048}^2,
    each from the ellipse recipe with its own 4-16 markers (FP32).  One pseudo-time step of all
    images to rho <= 1e-6 through the batch graph (one launch per V-cycle, converged images skipped
    on the device), tile shapes from the autotuner, against the same images solved one by one.
    Returns a dict."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    buildlib.build()
    dev = torch.device("cuda", dev_index)
    rng = np.random.Generator(np.random.PCG64(3))
    sizes = rng.choice([256, 512, 768, 1024, 2048], size=count)
    imgs, mks, params = [], [], []
    for q, n in enumerate(sizes):
        k = int(rng.integers(4, 17))
        img, mk = synth.ellipses_device(int(n), int(n), max(12, int(12 * n / 1024)),
                                        (20 * n / 1024, 200 * n / 1024), k, 0.05, 100 + q, dev)
        imgs.append(img)
        mks.append(mk)
        params.append(segmg.default_params(int(n), int(n)))
    cells = int(sum(int(n) ** 2 for n in sizes))

    def batch_run(tune, reps):
        # one untimed step (graph build, and the tuning when asked), then `reps` timed steps from
        # the same images (mg_reset of every image: tau back to its parameter, graphs kept)
        b = segmg.Batch(imgs, mks, params)
        if tune:
            b.autotune(reps=1)
        b.solve_step(TOL, MAX_CYCLES)
        out = []
        for _ in range(reps):
            b.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cyc, rho = b.solve_step(TOL, MAX_CYCLES)
            out.append((time.perf_counter() - t0, cyc, rho))
        b.close()
        return out

    tb = batch_run(True, max(1, steps))
    tb_plain = batch_run(False, max(1, steps))
    ts = []
    for _ in range(max(1, steps)):
        tot, cyc_s = 0.0, []
        for q in range(len(imgs)):
            s = segmg.Solver(imgs[q], mks[q], params[q])
            s.solve_step(TOL, MAX_CYCLES)      # warm-up / graph capture of this image
            s.reset(imgs[q], mks[q])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c, r = s.solve_step(TOL, MAX_CYCLES)
            tot += time.perf_counter() - t0
            cyc_s.append(c)
            s.close()
        ts.append(tot)
    best_b = min(tb, key=lambda x: x[0])
    return {"config": f"batched: {len(sizes)} FP32 images, sizes {sorted(set(int(x) for x in sizes))}",
            "size_counts": {int(k): int((sizes == k).sum()) for k in sorted(set(sizes))},
            "cells": cells,
            "batched_autotuned": {"s": best_b[0], "unknowns_per_s": cells / best_b[0],
                                  "cycles_min_max": [min(best_b[1]), max(best_b[1])],
                                  "rho_max": max(best_b[2])},
            "batched_default_tiles": {"s": min(x[0] for x in tb_plain),
                                      "unknowns_per_s": cells / min(x[0] for x in tb_plain),
                                      "rho_max": max(max(x[2]) for x in tb_plain)},
            "one_by_one": {"s": min(ts), "unknowns_per_s": cells / min(ts)},
            "speedup_batched_vs_one_by_one": min(ts) / best_b[0]}


def run_algorithms(args):
    """The paper's Algorithms 1, 2 and 3 on the GPU (Sec. 5, Tables 6-7 analogue on synthetic data):
    FAS with GSLINE-I, with Hybrid Smoother 1 and with Hybrid Smoother 2, one pseudo-time step
    from the initial contour to rho <= 1e-6 on an N x N ellipse image, at V(2,2) and at the
    paper's smoothing counts (5, 3, 3).  Reports V-cycles, the step's device time, rho and the
    level-set energy after each V-cycle (the Table 7 diagnostic)."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    buildlib.build()
    N = args.algorithms
    W = synth.workload(WORKLOAD) if N == 1024 else None
    img, mk = (W.image, W.markers) if W else synth.ellipses(
        N, N, max(12, 12 * N // 1024), (20 * N / 1024, 200 * N / 1024), 8, 0.05, 1)[:2]
    timg = torch.as_tensor(img.astype(np.float32), device="cuda")
    algos = [("Algorithm 1 (GSLINE-I)", segmg.MG_SMOOTH_GSLINE, 5),
             ("Algorithm 2 (Hybrid Smoother 1)", segmg.MG_SMOOTH_HS1, 3),
             ("Algorithm 3 (Hybrid Smoother 2)", segmg.MG_SMOOTH_FUSED, 3)]
    rows = []
    for name, sm, nu_paper in algos:
        for nu in (2, nu_paper):
            p = segmg.default_params(N, N, smoother=sm, nu1=nu, nu2=nu)
            s = segmg.Solver(timg, mk, p)
            st = torch.cuda.ExternalStream(s.stream_ptr)
            energies, rhos, ms = [], [], []
            for rep in range(2):          # the second run is timed (graph built, caches warm)
                s.reset(timg, mk)
                s.begin_step()
                energies, rhos, ms = [s.energy()], [], []
                for _ in range(MAX_CYCLES * 2):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    r = s.vcycle()
                    b.record(st)
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
                    rhos.append(r)
                    energies.append(s.energy())
                    if r <= TOL:
                        break
            rows.append({"algorithm": name, "nu1": nu, "nu2": nu, "cycles": len(rhos),
                         "converged": rhos[-1] <= TOL, "rho": rhos[-1], "ms_vcycles": float(sum(ms)),
                         "ms_per_cycle": float(np.mean(ms)), "energy": energies})
            s.close()
    # the AOS method of Table 6 on the same step: iterations to a relative change <= 1e-4 (the
    # paper's stop), the residual it reaches, its time
    for dt in (0.25, 1.0):
        p = segmg.default_params(N, N)
        s = segmg.Solver(timg, mk, p)
        st = torch.cuda.ExternalStream(s.stream_ptr)
        for rep in range(2):
            s.reset(timg, mk)
            s.begin_step()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            it, r = s.aos(dt, 2000, 1e-4)
            b.record(st)
            b.synchronize()
        rows.append({"algorithm": f"AOS (dt {dt})", "iterations": it, "rho": r, "eta_stop": 1e-4,
                     "ms": a.elapsed_time(b), "energy_end": s.energy()})
        s.close()
    print(json.dumps({"algorithms": N, "tol": TOL, "rows": rows}), flush=True)


def run_learned(args):
    print(json.dumps(learned_report(args.learned, args.loss, args.train_iters, args.refresh)), flush=True)


def learned_report(sizes, loss_kind="hf", train_iters=1000, refresh=4, dev_index=0):
    """Learned relaxation weights (the config-5 form): train on states recorded from 200 plain
    solves of 1024^2 ellipse images (seeds 100-299), then time one pseudo-time step to
    rho <= 1e-6 at the given sizes with the plain smoother and with the learned weights kept per
    V-cycle only when they beat the plain smoother's rate (mode 1)."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    buildlib.build()
    dev = torch.device("cuda", dev_index)
    t0 = time.perf_counter()
    tr = segmg.Trainer(capacity=200 * 24, batch_max=64, seed=5)
    tr.set_loss(loss_kind)
    for k in range(200):
        img, mk, _ = synth.ellipses(1024, 1024, 12, (20, 200), 8, 0.05, 100 + k)
        s = segmg.Solver(torch.as_tensor(img.astype(np.float32), device=dev), mk, segmg.default_params(1024, 1024))
        s.begin_step()
        for c in range(6):
            s.vcycle()
            if c in (0, 2, 5):
                tr.record(s, 8)
        s.close()
    t_rec = time.perf_counter() - t0
    loss0 = tr.grad(list(range(64)))[0]
    t1 = time.perf_counter()
    loss = tr.train(train_iters, 64, 3e-3)
    t_train = time.perf_counter() - t1
    loss1 = tr.grad(list(range(64)))[0]
    theta = tr.theta()
    rows = []
    for N in sizes:
        # the config-3 image recipe scaled to N (200 ellipses, axes 100-3000 px at 25000^2, the
        # device-side generator of the config-3 run)
        img, mk = synth.ellipses_device(N, N, 200, (100 * N / 25000, 3000 * N / 25000), 20, 0.05, 2, dev)
        img = img.float().cpu().numpy() if hasattr(img, "cpu") else img
        levels, sz = 1, N
        while sz // 2 >= 4 and levels < 12:
            sz //= 2
            levels += 1
        W = synth.Workload(f"ellipses200_{N}", img, mk, levels, TOL, "f32", "config-3 recipe")
        timg = torch.as_tensor(W.image.astype(np.float32), device=dev)
        for mode in (0, 1):
            p = segmg.default_params(N, N, levels=W.levels)
            s = segmg.Solver(timg, W.markers, p)
            if mode:
                s.set_learned(theta, mode=1, refresh=refresh)
            st = torch.cuda.ExternalStream(s.stream_ptr)
            for rep in range(2):                    # the second run is timed
                s.reset(timg, W.markers)
                a0 = s.stats()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                cyc, rho = s.solve_step(TOL, MAX_CYCLES)
                b.record(st)
                b.synchronize()
            stt = s.stats()
            rows.append({"n": N, "mode": "learned (per V-cycle acceptance)" if mode else "plain",
                         "cycles": cyc, "rho": rho, "converged": rho <= TOL, "ms": a.elapsed_time(b),
                         "unknowns_per_s": N * N / (a.elapsed_time(b) * 1e-3),
                         "learned_accepted": stt["learned_accepted"] - a0["learned_accepted"],
                         "learned_rejected": stt["learned_rejected"] - a0["learned_rejected"]})
            s.close()
    crops = tr.count
    tr.close()
    return {"learned": {"loss": loss_kind, "crops": crops, "record_s": t_rec, "train_iters": train_iters,
                        "train_s": t_train, "loss_before": loss0, "loss_after": loss1, "last_batch_loss": loss,
                        "refresh": refresh},
            "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hbm-roofline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 25000^2 and 64-image reports")
    ap.add_argument("--sample-cycles", type=int, default=0,
                    help="reference arm: V-cycles per sample (0: the whole step is timed)")
    ap.add_argument("--profile", type=int, default=0, help="run the N x N ncu profiling case instead")
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--tile-shape", type=int, default=-1, help="profiling case: this tile shape on every grid")
    ap.add_argument("--autotune", action="store_true", help="profiling case: mg_autotune first, as the bench")
    ap.add_argument("--shapes", default="", help="profiling case: tile shape per grid, comma-separated")
    ap.add_argument("--cluster-level", type=int, default=None, help="profiling case: first grid of the cluster bottom")
    ap.add_argument("--time-kernels", action="store_true",
                    help="profiling case: run mg_time_kernels and mg_time_residuals once on the finest grid first")
    ap.add_argument("--config3", type=int, default=0, help="run the mixed-precision N x N report")
    ap.add_argument("--config4", type=int, default=0, help="run the batched report with this many images")
    ap.add_argument("--algorithms", type=int, default=0, help="compare Algorithms 1-3 on an N x N image")
    ap.add_argument("--learned", type=int, nargs="*", default=None,
                    help="train the learned relaxation weights, then compare at these sizes")
    ap.add_argument("--train-iters", type=int, default=1000)
    ap.add_argument("--refresh", type=int, default=4)
    ap.add_argument("--loss", choices=["full", "hf"], default="full",
                    help="learned weights: train on the residual or on its high-frequency part")
    args = ap.parse_args()
    if args.learned is not None:
        if not args.learned:
            args.learned = [4096, 8192]
        run_learned(args)
    elif args.algorithms:
        run_algorithms(args)
    elif args.config4:
        run_config4(args)
    elif args.config3:
        run_config3(args)
    elif args.profile:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
