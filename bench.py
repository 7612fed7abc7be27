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
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = [r.split(",") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
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


def oracle_sample(img, mk, cycles_needed=None, full=False, sample_cycles=2):
    """Times the oracle on the workload: set-up, begin_step and `sample_cycles` V-cycles (all
    V-cycles to rho <= 1e-6 when `full`).  Returns a dict."""
    import oracle as O
    n, m = img.shape
    p = O.params(n, m, levels=9)
    t0 = time.perf_counter()
    s = O.Solver(img.astype(np.float64), mk, p)
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
    rank, ws, _, dist = dist_init()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    from paper_1807_02137_gb300 import synth
    W = synth.workload(WORKLOAD)
    img, mk = W.image, W.markers
    n, m = img.shape
    cycles_needed = None
    for w in range(args.warmup):
        r = oracle_sample(img, mk, full=(w == 0 and args.sample_cycles >= 2))
        if w == 0 and args.sample_cycles >= 2:
            cycles_needed = r["cycles_run"]
    if cycles_needed is None:
        cycles_needed = 13
    per_step = []
    for _ in range(args.steps):
        r = oracle_sample(img, mk, sample_cycles=args.sample_cycles)
        per_step.append(r["setup"] + r["begin"] + cycles_needed * r["cycle"])
    sec = float(np.mean(per_step))
    value = n * m / sec
    sample = (f"FP64 C oracle, 1 host core: set-up + begin_step + {args.sample_cycles} V-cycles of the {n}x{m} workload "
              f"per step, scaled to the {cycles_needed} V-cycles the oracle needs to reach rho <= 1e-6 "
              f"(measured in the first warm-up step)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{WORKLOAD}: {n}x{m} FP32 image, 12 ellipses, 8 markers, 9 grids, "
                                   f"V(2,2), tau 1, one pseudo-time step to rho <= 1e-6",
                       "l2": "n/a (host)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
        r = None
        try:
            r = oracle_sample(img_np, mk)     # before any GPU call
        except Exception as e:  # the baseline is a report, never a reason to fail the bench
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
        if r:
            cpu = r

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

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, cycles, rhos = [], [], []
    l0 = s.stats()["launches"]
    with Clocks(lrank) as clk:
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

    # end to end through the host-buffer entry point (copies inside the timed region)
    e2e_ms = []
    for k in range(0 if args.no_e2e else max(1, min(args.steps, 5)) + 1):
        t0 = time.perf_counter()
        segmg.segment_host(img_np, mk, p, TOL, MAX_CYCLES, 0.0, 1)
        if k > 0:
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
    sweep_ms = float(np.mean(kt[1:5]))
    bytes_per_cell = 16.125        # u, G, f (4 B each) + member masks (1/8 B) read, u (4 B) written
    achieved = bytes_per_cell * n * m / (sweep_ms * 1e-3) / 1e9
    # DRAM bytes of one finest-grid sweep launch from an ncu capture of this kernel on this grid
    # (profiles/k_sweep_tma_traffic_ellipse1024.txt): u, G, f read once, u written to L2
    traffic = 12.76e6
    roof = {"bound": "hbm", "kernel": "k_sweep_tma (TMA-staged fused Hybrid Smoother 2 sweep, finest grid)",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "peak_kind": peak_kind + " (hbm_gbs, burst copy)",
            "bytes_per_cell": bytes_per_cell, "ms_per_launch": sweep_ms,
            "note": "1024^2 working set is L2-resident inside a step; see roofline_hbm for 8192^2"}
    roof_big = None
    if not args.no_hbm_roofline:
        try:
            img8, mk8, _ = synth.ellipses(8192, 8192, 96, (160, 1600), 8, 0.05, 1)
            p8 = segmg.default_params(8192, 8192)
            s8 = segmg.Solver(torch.as_tensor(img8, device=dev), mk8, p8)
            s8.begin_step()
            kt8 = s8.time_kernels(0, reps=3)
            sw8 = float(np.mean(kt8[1:5]))
            ach8 = bytes_per_cell * 8192 * 8192 / (sw8 * 1e-3) / 1e9
            snap_bytes = 24.25       # pn, u, w, F read; G, f and member masks (1/4 B) written
            res_bytes = 16           # pn, u, w, F read, r written (+ 0 rhs on the finest grid)
            roof_big = {"bound": "hbm", "grid": "8192x8192 FP32", "unit": "GB/s", "peak": hbm,
                        "sweep": {"ms": sw8, "achieved": ach8, "frac": ach8 / hbm},
                        "snapshot": {"ms": kt8[0], "achieved": snap_bytes * 8192 ** 2 / (kt8[0] * 1e-3) / 1e9},
                        "residual": {"ms": kt8[5], "achieved": res_bytes * 8192 ** 2 / (kt8[5] * 1e-3) / 1e9}}
            for k in ("snapshot", "residual"):
                roof_big[k]["frac"] = roof_big[k]["achieved"] / hbm
            s8.close()
        except Exception as e:
            roof_big = {"error": str(e)}

    cpu_line = None
    if cpu and "setup" in cpu:
        cyc = float(np.mean(cycles))
        sec = cpu["setup"] + cpu["begin"] + cyc * cpu["cycle"]
        cpu_line = {"value": n * m / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": (f"FP64 C oracle on 1 host core: set-up + begin_step + 2 V-cycles of the same "
                               f"{n}x{m} workload ({cpu['setup'] + cpu['begin'] + 2 * cpu['cycle']:.1f} s), "
                               f"scaled to the {cyc:.1f} V-cycles per step the GPU needed")}
    elif cpu:
        cpu_line = cpu

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
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max,
                    "path": "mg_segment_host (host image in, host mask out; allocation and set-up included)"},
            "gpu_launches": int(launches),
            "roofline": roof, "roofline_hbm": roof_big,
            "cpu_baseline": cpu_line,
            "clocks": clk.summary(),
            "wall_s_timed_region": t_wall}
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
    for _ in range(args.cycles):
        r = s.vcycle()
    print(json.dumps({"profile_case": N, "cycles": args.cycles, "rho": r, **s.stats()}), flush=True)
    s.close()


def run_config3(args):
    """Mixed precision at large size (w stored in BF16, smoothing FP32, FP64 norms and coarsest
    solve): one pseudo-time step to rho <= 1e-6 on an N x N image from the ellipse recipe
    (200 ellipses, axes 100-3000 px, 20 markers), the smoother roofline at that size, and the
    error against the FP64 oracle on a 2048 x 2048 crop solved as a standalone problem."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    import oracle as O
    buildlib.build()
    N = args.config3
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    img, mk = synth.ellipses_device(N, N, 200, (100 * N / 25000, 3000 * N / 25000), 20, 0.05, 2, dev)
    gen_s = time.perf_counter() - t0
    p = segmg.default_params(N, N, precision=segmg.MG_MIXED)
    s = segmg.Solver(img, mk, p)
    st = torch.cuda.ExternalStream(s.stream_ptr, device=dev)
    s.solve_step(TOL, MAX_CYCLES)                 # warm-up (graph capture)
    times, cyc = [], []
    with Clocks(0) as clk:
        for _ in range(max(1, args.steps)):
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
    C = min(2048, N)
    cx, cy = float(np.mean(mk[:, 0])), float(np.mean(mk[:, 1]))
    j0 = int(min(max(cx - C / 2, 0), N - C)); i0 = int(min(max(cy - C / 2, 0), N - C))
    crop = img[i0:i0 + C, j0:j0 + C].float().cpu().numpy().copy()
    cmk = mk - np.array([j0, i0])
    cmk = cmk[(cmk[:, 0] >= 0) & (cmk[:, 0] <= C - 1) & (cmk[:, 1] >= 0) & (cmk[:, 1] <= C - 1)]
    del img
    torch.cuda.empty_cache()
    out = {}
    for name, prec in (("mixed", segmg.MG_MIXED), ("f32", segmg.MG_F32)):
        pc = segmg.default_params(C, C, precision=prec)
        sc = segmg.Solver(torch.as_tensor(crop, device=dev), cmk, pc)
        sc.solve_step(TOL, MAX_CYCLES)
        out[name] = sc.phi().double().cpu().numpy()
        sc.close()
    po = O.params(C, C, levels=segmg.default_params(C, C).levels)
    t1 = time.perf_counter()
    so = O.Solver(crop.astype(np.float64), cmk, po)
    hist = so.solve_step(1e-9, 80)
    ref = so.phi
    oracle_s = time.perf_counter() - t1
    acc = {}
    for name, phi in out.items():
        acc[name] = {"max_rel_err_phi": float(np.max(np.abs(phi - ref)) / np.max(np.abs(ref))),
                     "mask_mismatch_frac": float(np.mean((phi > 0) != (ref > 0)))}
    line = {"config": f"{N}x{N} mixed precision (w BF16, smoothing FP32, FP64 norms/coarsest)",
            "levels": stats["levels"], "unknowns_per_s": N * N / (np.mean(times) * 1e-3),
            "ms_per_step": float(np.mean(times)), "cycles_per_step": float(np.mean(cyc)),
            "device_bytes": stats["device_bytes"], "generate_s": gen_s,
            "roofline_sweep": {"ms": sw, "achieved_GBs": 16.125 * N * N / (sw * 1e-3) / 1e9, "peak": hbm,
                               "frac": 16.125 * N * N / (sw * 1e-3) / 1e9 / hbm},
            "kernel_ms": {"snapshot": kt[0], "sweeps": kt[1:5], "residual": kt[5]},
            "crop": {"size": C, "origin": [i0, j0], "markers": int(len(cmk)), "oracle_cycles": len(hist),
                     "oracle_rho": hist[-1], "oracle_s": oracle_s, **acc},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_config4(args):
    """Batched uneven sizes: 64 images with sizes drawn from {256, 512, 768, 1024, 2048}^2, each
    from the ellipse recipe with its own 4-16 markers (FP32).  One pseudo-time step of all images
    to rho <= 1e-6 through the batch graph (one launch per V-cycle, converged images skipped on
    the device), tile shapes from the autotuner, against the same images solved one by one."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    buildlib.build()
    dev = torch.device("cuda", 0)
    rng = np.random.Generator(np.random.PCG64(3))
    sizes = rng.choice([256, 512, 768, 1024, 2048], size=args.config4)
    imgs, mks, params = [], [], []
    for q, n in enumerate(sizes):
        k = int(rng.integers(4, 17))
        img, mk = synth.ellipses_device(int(n), int(n), max(12, int(12 * n / 1024)),
                                        (20 * n / 1024, 200 * n / 1024), k, 0.05, 100 + q, dev)
        imgs.append(img)
        mks.append(mk)
        params.append(segmg.default_params(int(n), int(n)))
    cells = int(sum(int(n) ** 2 for n in sizes))

    def batch_run(tune):
        b = segmg.Batch(imgs, mks, params)
        shapes = None
        if tune:
            b.autotune(reps=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc, rho = b.solve_step(TOL, MAX_CYCLES)
        dt = time.perf_counter() - t0
        b.close()
        return dt, cyc, rho

    batch_run(True)                       # warm-up (graph build, autotune, caches)
    tb = [batch_run(True) for _ in range(max(1, args.steps))]
    tb_plain = [batch_run(False) for _ in range(max(1, args.steps))]
    ts = []
    for _ in range(max(1, args.steps)):
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
    line = {"config": f"batched: {len(sizes)} FP32 images, sizes {sorted(set(int(x) for x in sizes))}",
            "size_counts": {int(k): int((sizes == k).sum()) for k in sorted(set(sizes))},
            "cells": cells,
            "batched_autotuned": {"s": best_b[0], "unknowns_per_s": cells / best_b[0],
                                  "cycles_min_max": [min(best_b[1]), max(best_b[1])],
                                  "rho_max": max(best_b[2])},
            "batched_default_tiles": {"s": min(x[0] for x in tb_plain),
                                      "unknowns_per_s": cells / min(x[0] for x in tb_plain)},
            "one_by_one": {"s": min(ts), "unknowns_per_s": cells / min(ts)},
            "speedup_batched_vs_one_by_one": min(ts) / best_b[0]}
    print(json.dumps(line), flush=True)


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
    """Learned relaxation weights (the config-5 form): train on states recorded from 200 plain
    solves of 1024^2 ellipse images (seeds 100-299), then time one pseudo-time step to
    rho <= 1e-6 at the given sizes with the plain smoother and with the learned weights kept per
    V-cycle only when they beat the plain smoother's rate (mode 1)."""
    import torch
    from paper_1807_02137_gb300 import buildlib, segmg, synth
    buildlib.build()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    tr = segmg.Trainer(capacity=200 * 24, batch_max=64, seed=5)
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
    loss = tr.train(args.train_iters, 64, 3e-3)
    t_train = time.perf_counter() - t1
    loss1 = tr.grad(list(range(64)))[0]
    theta = tr.theta()
    rows = []
    for N in args.learned:
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
                s.set_learned(theta, mode=1, refresh=args.refresh)
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
    print(json.dumps({"learned": {"crops": tr.count, "record_s": t_rec, "train_iters": args.train_iters,
                                  "train_s": t_train, "loss_before": loss0, "loss_after": loss1,
                                  "last_batch_loss": loss, "refresh": args.refresh},
                      "rows": rows}), flush=True)
    tr.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hbm-roofline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sample-cycles", type=int, default=2, help="V-cycles per reference-arm sample")
    ap.add_argument("--profile", type=int, default=0, help="run the N x N ncu profiling case instead")
    ap.add_argument("--cycles", type=int, default=2)
    ap.add_argument("--tile-shape", type=int, default=-1, help="profiling case: this tile shape on every grid")
    ap.add_argument("--config3", type=int, default=0, help="run the mixed-precision N x N report")
    ap.add_argument("--config4", type=int, default=0, help="run the batched report with this many images")
    ap.add_argument("--algorithms", type=int, default=0, help="compare Algorithms 1-3 on an N x N image")
    ap.add_argument("--learned", type=int, nargs="*", default=None,
                    help="train the learned relaxation weights, then compare at these sizes")
    ap.add_argument("--train-iters", type=int, default=1000)
    ap.add_argument("--refresh", type=int, default=4)
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
