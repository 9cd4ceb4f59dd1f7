#!/usr/bin/env python
"""Benchmark of the GB300 PDHG photoacoustic reconstruction.

Metric: PDHG iterations per second of the TGV^2 reconstruction of a 256^2 vessel phantom
from 256 detectors x 512 time samples (M = 256 quadrature points per circle, alpha 0.02,
beta 0.04, 1000 iterations per reconstruction, FP64 duality gap every 10 iterations).

One step = one full reconstruction through the C ABI (pat_reconstruct): step sizes,
initialisation, 1000 PDHG iterations with gap evaluations, output.  Inputs are resident
in HBM when the step starts; the L2 cache is flushed before every step (a 256 MiB write
outside the timed events).  Each rank of a multi-GPU run solves its own independent
problem (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

``--impl reference`` times the FP64 CPU oracle (the reference of this build) on the host
cores for the same workload and metric, one oracle PDHG iteration per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PDHG iters/sec (TGV^2 256x256, 256 det x 512 samples)"
UNIT = "iters/s"
WORKLOAD_DESC = ("tgv256: TGV^2 PDHG, 256x256 vessel phantom with exp(-3 depth) fluence, 256 detectors on a "
                 "full circle r=1.2, 512 time samples, M=256, 5% noise, alpha 0.02, beta 0.04, 1000 iterations, "
                 "diagonal preconditioning, FP64 gap every 10 iterations")
# Algorithmic work of one quadrature point of K or K^T: about 15 FP32 operations
# (position 2 FMA, floor and fraction 4, bilinear weights and lerps 8, accumulate 1) and
# 4 gathered (K) or scattered (K^T) taps.  The projector bound is the smaller of the FP32
# issue rate over 15 and the load/store rate over 4 (per SM and clock: 128 FP32 lanes,
# 32 shared or L1 lane accesses).
OPS_PER_POINT, TAPS_PER_POINT = 15, 4
FP32_LANES, LSU_LANES = 128, 32


# ---------------------------------------------------------------------------------
# distributed helpers (host logic; tested with gloo on CPU)
# ---------------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(dist, seconds: float, units: float, device=None) -> tuple[float, float]:
    """(max seconds over ranks, summed units over ranks)."""
    if dist is None:
        return seconds, units
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------------
# clocks sampler
# ---------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------

def oracle_setup(workload: str, seed: int, workers: int):
    """Oracle problem for the workload (data simulated with the oracle on the same grid),
    with K and K^T applied over ``workers`` host processes (detector subsets)."""
    import numpy as np

    import synthetic as S
    from oracle import pat_oracle as O
    from oracle.parallel import OraclePool
    w = S.workload(workload, seed)
    g = O.Geometry(n=w["n"], det_xy=w["det_xy"], n_t=w["n_t"], r0=w["r0"], dr=w["dr"], quad_m=w["quad_m"])
    pool = OraclePool(g, workers)
    clean = pool.forward(w["phantom"])
    f = clean + w["noise_level"] * np.abs(clean).max() * w["noise"]
    xi = O.direction_field(w["side"], w["eta"]) if w["reg"] == O.REG_DTV else None
    pb = pool.problem(f, reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi)
    return pb, O.diag_steps(pb), pool


def oracle_iters_per_s(pb, steps, iters: int) -> tuple[float, float]:
    from oracle import pat_oracle as O
    t0 = time.perf_counter()
    O.pdhg(pb, iters, steps=steps, gap_every=0, final_gap=False)
    dt = time.perf_counter() - t0
    return iters / dt, dt


def oracle_baseline(workload: str, iters: int) -> dict:
    """The FP64 oracle's PDHG iterations/s on all host cores (K and K^T over detector
    subsets in worker processes) and on one core; setup untimed."""
    from oracle.parallel import host_cores
    cores = host_cores()
    out = {}
    for key, workers in (("all", cores), ("one", 1)):
        pb, st, pool = oracle_setup(workload, 0, workers)
        try:
            oracle_iters_per_s(pb, st, 1) if workers > 1 else None     # start the workers
            it_s, dt = oracle_iters_per_s(pb, st, iters)
        finally:
            pool.close()
        out[key] = {"value": it_s, "cores": len(pool.spans), "seconds": dt}
    return out


# ---------------------------------------------------------------------------------
# reference arm
# ---------------------------------------------------------------------------------

def run_reference(args) -> int:
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle.parallel import host_cores
    pb, st, pool = oracle_setup(args.workload, 0, host_cores())
    try:
        for _ in range(args.warmup):
            oracle_iters_per_s(pb, st, 1)
        times = []
        for _ in range(args.steps):
            _, dt = oracle_iters_per_s(pb, st, 1)
            times.append(dt)
    finally:
        pool.close()
    total = sum(times)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "iters_per_step": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(pool.spans), "kind": "oracle",
                             "sample": "one FP64 oracle PDHG iteration of the tgv256 workload per step "
                                       "(matrix-free numpy K and K^T over detector subsets on all host cores)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------------

def run_gb300(args) -> int:
    import numpy as np
    import torch

    import __graft_entry__
    import paper_1707_02245_gb300 as P
    import synthetic as S

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    dist = init_dist(world, "nccl")
    __graft_entry__.build()
    stream = torch.cuda.current_stream(device)

    # ---- inputs (seeded; each rank solves its own problem) ----
    w = S.workload(args.workload, seed=rank)
    n = w["n"]
    fine = P.Geometry(w["n_fine"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m_fine"])
    ph_f = torch.from_numpy(w["phantom_fine"].astype(np.float32)).to(device)
    clean = torch.empty(w["det_xy"].shape[0], w["n_t"], device=device)
    P.pat_forward(fine.handle, ph_f, clean, stream)
    noise = torch.from_numpy(w["noise"].astype(np.float32)).to(device)
    f = (clean + w["noise_level"] * clean.abs().max() * noise).contiguous()
    fine.close()
    geo = P.Geometry(n, w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    ginfo = geo.info()
    xi = None
    if w["reg"] == P.PAT_DTV:
        side = torch.from_numpy(w["side"].astype(np.float32)).to(device)
        xi = torch.empty(2, n, n, device=device)
        P.pat_direction_field(n, side, w["eta"], xi, stream)
    u = torch.empty(n, n, device=device)
    iters = args.iters or w["iters"]
    prm = P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi,
                        iters=iters, gap_every=10, tol=0.0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    # ---- launch shapes chosen by the library's autotuner (one-off, before the timed steps)
    shapes = None
    cache = SHAPE_CACHE[0] = None if args.no_tune else (
        args.shape_cache or os.path.join(tempfile.mkdtemp(prefix="pat_shapes_"), "shapes.json"))
    if cache:
        t0 = time.perf_counter()
        chosen = P.pat_tune_shapes([geo.handle], [f], [prm], reps=50, cache_path=cache, stream=stream)
        shapes = {"chosen": chosen[0], "tune_seconds": time.perf_counter() - t0,
                  "timed_us": next((e["us"] for e in json.load(open(cache))["entries"]
                                    if e["key"].startswith("N=%d D=%d T=%d " % (n, w["det_xy"].shape[0], w["n_t"]))),
                                   None),
                  "how": "pat_tune_shapes: K variants, K^T waves (1, 2), update tiles (32x4, 32x8, 64x4), "
                         "each timed in a CUDA graph of 50 launches on this problem; fastest kept"}
    else:
        shapes = {"chosen": P.pat_geometry_get_shapes(geo.handle), "tune_seconds": None}

    def step():
        return P.pat_reconstruct(geo.handle, f, prm, u, stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize(device)

    # ---- timed region: K steps, per-step CUDA events, per-phase profiling on ----
    sampler = ClockSampler(device.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(dist, device)
    torch.cuda.synchronize(device)
    sampler.start()
    launches0 = P.pat_kernel_launches()

    def timed_steps(k):
        ms, inf = [], []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inf.append(step())
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, inf

    wall0 = time.perf_counter()
    step_ms, infos = timed_steps(args.steps)
    torch.cuda.synchronize(device)
    wall = time.perf_counter() - wall0
    launches = P.pat_kernel_launches() - launches0
    barrier(dist, device)
    # per-launch device time of each phase: every phase captured alone in a CUDA graph of
    # 200 launches after 100 iterations of the same problem, replayed between CUDA events
    prm_ph = P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi,
                           iters=100, gap_every=10)
    phase_us = P.pat_time_phases([geo.handle], [f], [prm_ph], 200, stream)
    clocks = sampler.stop()

    local_s = sum(step_ms) / 1e3
    max_s, units = aggregate(dist, local_s, float(iters * args.steps), device)
    value = units / max_s

    # ---- end to end through the public call with host buffers ----
    f_host = f.cpu().pin_memory()
    u_host = torch.empty(n, n).pin_memory()
    f_dev = torch.empty_like(f)
    prm_e2e = P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi,
                            iters=iters, gap_every=10, tol=0.0)
    e2e_ms = []
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 5))
    for _ in range(e2e_steps + 1 if e2e_steps else 0):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f_dev.copy_(f_host, non_blocking=True)
        P.pat_reconstruct(geo.handle, f_dev, prm_e2e, u, stream)
        u_host.copy_(u, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e = None
    if e2e_steps:
        e2e_ms = e2e_ms[1:]
        e2e_s, e2e_units = aggregate(dist, sum(e2e_ms) / 1e3, float(iters * e2e_steps), device)
        e2e = {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": f.numel() * 4,
               "d2h_bytes_per_step": u.numel() * 4, "steps": e2e_steps}

    # ---- time to relative gap 1e-4 (cold start): the paper's steps, and the balance s
    # chosen by the probe tuner (probe time included) ----
    ttg = None
    if not args.no_ttg:
        def to_gap(ratio):
            prm_t = P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi,
                                  iters=args.ttg_max_iters, gap_every=10, tol=1e-4, step_ratio=ratio)
            flush.zero_()
            return P.pat_reconstruct(geo.handle, f, prm_t, u, stream)
        info = to_gap(1.0)
        ttg = {"tol": 1e-4, "paper_steps": {"step_ratio": 1.0, "iters": info["iters_done"],
                                            "seconds": info["ms"] / 1e3, "rel_gap": info["rel_gap"],
                                            "reached": info["status"] == P.PAT_STATUS_CONVERGED},
               "max_iters": args.ttg_max_iters}
        cands = [1.0, 3.0, 10.0, 30.0]
        prm_p = P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=xi)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        best, pg = P.pat_tune_step_ratio(geo.handle, f, prm_p, cands, args.probe_iters, stream)
        e1.record(stream)
        e1.synchronize()
        probe_s = e0.elapsed_time(e1) / 1e3
        info = to_gap(best)
        ttg["tuned"] = {"step_ratio": best, "candidates": cands, "probe_iters": args.probe_iters,
                        "probe_rel_gaps": pg, "probe_seconds": probe_s, "iters": info["iters_done"],
                        "solve_seconds": info["ms"] / 1e3, "seconds": probe_s + info["ms"] / 1e3,
                        "rel_gap": info["rel_gap"], "reached": info["status"] == P.PAT_STATUS_CONVERGED}
        ttg["speedup_vs_paper_steps"] = ttg["paper_steps"]["seconds"] / ttg["tuned"]["seconds"]

    # ---- the wavelet model (PAT_WAV) on the same data: iterations/s and time to gap ----
    wav = None
    if not args.no_wavelet:
        wav = run_wavelet_leg(P, torch, geo, f, u, stream, flush, args)

    # ---- measurement pre-processing (Sec. 4.3) on this geometry ----
    prep = None
    if not args.no_prep:
        prep = run_preprocess(P, S, np, torch, device, stream, geo, w, flush)

    # ---- batched: B TGV 256^2 problems in lockstep, and the 64-problem mixed batch ----
    batched = None
    if args.batch > 0:
        batched = run_batched_tgv(P, S, np, torch, device, stream, args.batch, iters, flush)
    mixed = None
    if args.mixed:
        mixed = run_mixed(P, S, np, torch, device, stream, flush, args.mixed_max_iters)
    upd_hbm = None
    if not args.no_update_hbm:
        upd_hbm = run_update_hbm(P, S, np, torch, device, stream, flush)
    warm = None
    if args.warm:
        warm = run_warm_start(P, S, np, torch, device, stream, args)

    # ---- roofline of the dominant phase ----
    NN = n * n
    pts = ginfo["points_on_grid"]
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peaks = load_peaks()
    f_max = (clocks.get("sm_max_mhz") or peaks["sm_max_mhz"]) * 1e6
    fp32_pts = sms * FP32_LANES * f_max / OPS_PER_POINT        # points/s at full FP32 issue
    lsu_pts = sms * LSU_LANES * f_max / TAPS_PER_POINT         # points/s at full load/store rate
    proj_peak = min(fp32_pts, lsu_pts)
    per_pixel_floats = {0: 8, 1: 18, 2: 10}[w["reg"]]
    per_step = {"forward_prox": iters, "adjoint": iters, "update": iters, "gap": iters // 10}
    phases = {}
    for ph, cnt in per_step.items():
        us = phase_us.get(ph) or 0.0
        if cnt == 0 or us <= 0:
            continue
        ent = {"avg_us": us, "launches_per_step": cnt, "share": None}
        if ph in ("forward_prox", "adjoint"):
            rate = pts / (us * 1e-6)
            ent.update(bound="alu", achieved=rate / 1e9, peak=proj_peak / 1e9, unit="Gpoint/s",
                       frac=rate / proj_peak, fp32_issue_frac=rate / fp32_pts, lsu_frac=rate / lsu_pts)
        elif ph == "update":
            gbs = 4.0 * per_pixel_floats * NN / (us * 1e-6) / 1e9
            ent.update(bound="hbm", achieved=gbs, peak=peaks["hbm_gbs"], unit="GB/s", frac=gbs / peaks["hbm_gbs"])
        phases[ph] = ent
    tot = sum(v["avg_us"] * v["launches_per_step"] for v in phases.values())
    for v in phases.values():
        v["share"] = v["avg_us"] * v["launches_per_step"] / tot if tot else None
    dom_name = max(("forward_prox", "adjoint", "update"), key=lambda k: phases[k]["share"] if k in phases else -1)
    dom = phases[dom_name]
    roofline = {"kernel": dom_name, "bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                "unit": dom["unit"], "frac": dom["frac"], "traffic": None,
                "measured": "pat_time_phases: the phase alone in a CUDA graph of 200 launches, CUDA events on its "
                            "stream, after 100 iterations of the benchmark problem",
                "peak_source": (f"min(FP32 issue / {OPS_PER_POINT}, load-store lanes / {TAPS_PER_POINT}) per "
                                f"quadrature point: {sms} SMs x min({FP32_LANES}/{OPS_PER_POINT}, "
                                f"{LSU_LANES}/{TAPS_PER_POINT}) x {f_max / 1e6:.0f} MHz")
                if dom["bound"] == "alu" else peaks["source"]}
    phase_ms_per_step = tot / 1e3

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ob = oracle_baseline(args.workload, args.cpu_iters)
        cpu = {"value": ob["all"]["value"], "unit": UNIT, "cores": ob["all"]["cores"], "kind": "oracle",
               "sample": f"{args.cpu_iters} FP64 oracle PDHG iteration(s) of the same workload, K and K^T over "
                         f"detector subsets on {ob['all']['cores']} worker processes ({ob['all']['seconds']:.1f} s; "
                         f"setup untimed)",
               "single_core": {"value": ob["one"]["value"], "unit": UNIT, "cores": 1,
                               "sample": f"the same iterations on one core ({ob['one']['seconds']:.1f} s)"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * max_s / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD_DESC, "iters_per_step": iters, "parallelism": f"replicas{world}",
                           "l2": "flushed before every step (256 MiB write outside the timed events)",
                           "points_on_grid_per_K": pts, "final_rel_gap": infos[-1]["rel_gap"]},
                "roofline": roofline, "phases": phases, "phase_ms_per_step": phase_ms_per_step, "shapes": shapes,
                "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "time_to_gap": ttg,
                "batched": batched, "mixed_batch": mixed, "warm_start": warm, "preprocess": prep, "wavelet": wav,
                "update_hbm": upd_hbm,
                "wall_s_timed": wall}
        print(json.dumps(line), flush=True)
    geo.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def make_problem(P, np, torch, device, stream, w):
    """Geometry, data (K on the 2x finer grid plus the recipe's noise) and parameters."""
    n = w["n"]
    fine = P.Geometry(w["n_fine"], w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m_fine"])
    ph_f = torch.from_numpy(w["phantom_fine"].astype(np.float32)).to(device)
    clean = torch.empty(w["det_xy"].shape[0], w["n_t"], device=device)
    P.pat_forward(fine.handle, ph_f, clean, stream)
    noise = torch.from_numpy(w["noise"].astype(np.float32)).to(device)
    f = (clean + w["noise_level"] * clean.abs().max() * noise).contiguous()
    fine.close()
    geo = P.Geometry(n, w["det_xy"], w["n_t"], w["r0"], w["dr"], w["quad_m"])
    xi = None
    if w["reg"] == P.PAT_DTV:
        side = torch.from_numpy(w["side"].astype(np.float32)).to(device)
        xi = torch.empty(2, n, n, device=device)
        P.pat_direction_field(n, side, w["eta"], xi, stream)
    u = torch.empty(n, n, device=device)
    return geo, f, xi, u


SHAPE_CACHE = [None]
UPDATE_MOVED_TGV = 92   # bytes per pixel the TGV update kernel reads and writes


def tune(P, geos, fs, prms, reps, stream):
    """Launch shapes of a set of problems by the library's autotuner, through the cache file
    of this benchmark run (problems whose geometry key was seen before take the cached
    shapes without timing).  Returns (chosen shapes, seconds), or the current shapes and
    None under --no-tune."""
    if SHAPE_CACHE[0] is None:
        return [P.pat_geometry_get_shapes(g) for g in geos], None
    t0 = time.perf_counter()
    chosen = P.pat_tune_shapes(geos, fs, prms, reps=reps, cache_path=SHAPE_CACHE[0], stream=stream)
    return chosen, time.perf_counter() - t0


def run_update_hbm(P, S, np, torch, device, stream, flush, count=16, n=512, iters=40):
    """The fused update (k_update_b) where its state does not fit in L2: a lockstep batch
    of ``count`` TGV^2 problems of n x n (vessel phantoms, 128 detectors, T = 2n), ``iters``
    iterations, the update timed alone in a CUDA graph.  Bytes per pixel: the algorithmic
    72 (18 floats: read u, v2, r2, s3, tau; write u, v2, r2, s3, ubar) and the 92 the
    kernel moves (besides: read K^T q and clear the next iteration's buffer, 8 bytes; read
    and write the bfloat16 low words of u, v2, 12 bytes)."""
    ws = [S.workload_warm(700000 + s, n=n, n_det=128) for s in range(count)]
    probs = [make_problem(P, np, torch, device, stream, w) for w in ws]
    prms = [P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], iters=iters, gap_every=10) for w in ws]
    geos, fs, us = [p[0].handle for p in probs], [p[1] for p in probs], [p[3] for p in probs]
    P.pat_reconstruct_batched(geos, fs, prms, us, stream)        # warm-up (K sums, kernels)
    # launch shapes by the autotuner: the 16 geometries share one key, so one is timed and
    # the others take its shapes from the cache
    chosen, tune_s = tune(P, geos, fs, prms, 20, stream)
    px = count * n * n
    peaks = load_peaks()
    out = {"problems": count, "n": n, "pixels": px, "state_bytes": UPDATE_MOVED_TGV * px}
    # (an NVTX range, so that a profiler can select this leg's launches)
    torch.cuda.nvtx.range_push("update_hbm_phases")
    phase_us = P.pat_time_phases(geos, fs, prms, 20, stream)
    torch.cuda.nvtx.range_pop()
    avg_s = phase_us["update"] * 1e-6
    alg = 18 * 4 * px / avg_s / 1e9
    moved = UPDATE_MOVED_TGV * px / avg_s / 1e9
    out.update({"avg_us": avg_s * 1e6,
                "roofline": {"bound": "hbm", "achieved": alg, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": alg / peaks["hbm_gbs"], "bytes_per_pixel": 72},
                "moved_gb_per_s": moved, "moved_frac": moved / peaks["hbm_gbs"], "moved_bytes_per_pixel": UPDATE_MOVED_TGV,
                "measured": "pat_time_phases: 20 launches in a CUDA graph after the batch's iterations",
                "phases_us": phase_us, "shapes": chosen[0], "tune_seconds": tune_s})
    for p in probs:
        p[0].close()
    return out


def run_batched_tgv(P, S, np, torch, device, stream, count, iters, flush):
    """count TGV 256^2 problems (seeds 0..count-1) in one lockstep pat_reconstruct_batched."""
    probs = [make_problem(P, np, torch, device, stream, S.workload("tgv256", seed=s)) for s in range(count)]
    w0 = S.workload("tgv256", 0)
    prms = [P.make_params(reg=w0["reg"], alpha=w0["alpha"], beta=w0["beta"], iters=iters, gap_every=10)
            for _ in probs]
    geos, fs, us = [p[0].handle for p in probs], [p[1] for p in probs], [p[3] for p in probs]
    chosen, tune_s = tune(P, geos, fs, prms, 50, stream)
    for _ in range(2):
        P.pat_reconstruct_batched(geos, fs, prms, us, stream)
    ms = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.pat_reconstruct_batched(geos, fs, prms, us, stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    for p in probs:
        p[0].close()
    t = sum(ms) / len(ms) / 1e3
    return {"problems": count, "iters_per_problem": iters, "ms_per_batch": 1e3 * t,
            "value": count * iters / t, "unit": "problem-iters/s", "shapes": chosen[0], "tune_seconds": tune_s}


def run_mixed(P, S, np, torch, device, stream, flush, max_iters):
    """The 64-problem mixed batch solved to relative gap 1e-4 (gap every 10 iterations)."""
    ws = S.workload_batch(0, 64)
    probs = [make_problem(P, np, torch, device, stream, w) for w in ws]
    prms = [P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=p[2],
                          iters=max_iters, gap_every=10, tol=1e-4) for w, p in zip(ws, probs)]
    geos, fs, us = [p[0].handle for p in probs], [p[1] for p in probs], [p[3] for p in probs]
    # warm-up: computes the K sums of every geometry and loads the kernels
    P.pat_reconstruct_batched(geos, fs, [P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"],
                                                       gamma=w["gamma"], xi=p[2], iters=20, gap_every=10)
                                         for w, p in zip(ws, probs)], us, stream)
    chosen, tune_s = tune(P, geos, fs, prms, 20, stream)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = P.pat_reconstruct_batched(geos, fs, prms, us, stream)
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    its = [i["iters_done"] for i in infos]
    conv = sum(1 for i in infos if i["status"] == P.PAT_STATUS_CONVERGED)
    out = {"problems": len(ws), "seconds": t, "converged": conv, "tol": 1e-4, "max_iters": max_iters,
           "iters_median": float(np.median(its)), "iters_max": int(max(its)),
           "problem_iters_per_s": sum(its) / t, "step_ratio": 1.0, "tune_seconds": tune_s,
           "shapes_used": sorted({(c["forward"], c["adjoint_waves"], c["update_tile"]) for c in chosen}),
           "pixels": int(sum(w["n"] ** 2 for w in ws)), "samples": int(sum(w["det_xy"].shape[0] * w["n_t"] for w in ws))}
    # the TGV problems with the balance picked by the batched probe tuner (TV and dTV keep
    # s = 1: short probes overshoot for them); probe time included
    tg = [k for k, w in enumerate(ws) if w["reg"] == P.PAT_TGV]
    e0.record(stream)
    best, _ = P.pat_tune_step_ratio_batched([geos[k] for k in tg], [fs[k] for k in tg], [prms[k] for k in tg],
                                            [1.0, 3.0, 10.0, 30.0], 300, stream)
    e1.record(stream)
    e1.synchronize()
    probe_s = e0.elapsed_time(e1) / 1e3
    ratio = [1.0] * len(ws)
    for k, b in zip(tg, best):
        ratio[k] = b
    prms2 = [P.make_params(reg=w["reg"], alpha=w["alpha"], beta=w["beta"], gamma=w["gamma"], xi=p[2],
                           iters=max_iters, gap_every=10, tol=1e-4, step_ratio=r) for w, p, r in zip(ws, probs, ratio)]
    flush.zero_()
    e0.record(stream)
    infos2 = P.pat_reconstruct_batched(geos, fs, prms2, us, stream)
    e1.record(stream)
    e1.synchronize()
    t2 = e0.elapsed_time(e1) / 1e3
    its2 = [i["iters_done"] for i in infos2]
    out["tuned_tgv"] = {"probe_seconds": probe_s, "seconds": t2 + probe_s, "solve_seconds": t2,
                        "converged": sum(1 for i in infos2 if i["status"] == P.PAT_STATUS_CONVERGED),
                        "converged_tgv": sum(1 for k in tg if infos2[k]["status"] == P.PAT_STATUS_CONVERGED),
                        "converged_tgv_paper_steps": sum(1 for k in tg if infos[k]["status"] == P.PAT_STATUS_CONVERGED),
                        "tgv_problems": len(tg), "iters_median": float(np.median(its2)),
                        "tgv_iters_median": float(np.median([its2[k] for k in tg])),
                        "tgv_iters_median_paper_steps": float(np.median([its[k] for k in tg])),
                        "step_ratios_tgv": best}
    for p in probs:
        p[0].close()
    return out


def run_wavelet_leg(P, torch, geo, f, u, stream, flush, args):
    """PAT_WAV (Sec. 2.2, alpha 0.02, 4 levels) on the benchmark's geometry and data, with the
    paper's dual-tree complex wavelet transform and with the orthonormal DWT: 1000 fixed
    iterations (gap every 10), then the time to rel gap 1e-4 with the paper's steps and with
    the probe-tuned balance (probe time included), and 1000 iterations of a lockstep batch of
    copies of the problem."""
    def leg(kind):
        def run(iters, tol, ratio):
            prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=iters, tol=tol, gap_every=10, wavelet_levels=4,
                                step_ratio=ratio, wavelet_kind=kind)
            flush.zero_()
            return P.pat_reconstruct(geo.handle, f, prm, u, stream)
        run(50, 0.0, 1.0)
        fixed = run(1000, 0.0, 1.0)
        out = {"alpha": 0.02, "levels": 4, "iters_per_s": 1000 / (fixed["ms"] / 1e3), "ms_per_1000_iters": fixed["ms"]}
        if args.wavelet_batch > 1:
            # B copies of the problem as one lockstep batch: 1000 iterations each
            B = args.wavelet_batch
            us = [torch.empty_like(u) for _ in range(B)]
            prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=50, gap_every=10, wavelet_levels=4, wavelet_kind=kind)
            P.pat_reconstruct_batched([geo.handle] * B, [f] * B, [prm] * B, us, stream)
            prm = P.make_params(reg=P.PAT_WAV, alpha=0.02, iters=1000, gap_every=10, wavelet_levels=4, wavelet_kind=kind)
            flush.zero_()
            ms = P.pat_reconstruct_batched([geo.handle] * B, [f] * B, [prm] * B, us, stream)[0]["ms"]
            out["batched"] = {"problems": B, "problem_iters_per_s": B * 1000 / (ms / 1e3), "ms_per_1000_iters": ms}
        paper = run(args.ttg_max_iters, 1e-4, 1.0)
        out["time_to_gap_paper_steps"] = {"iters": paper["iters_done"], "seconds": paper["ms"] / 1e3,
                                          "reached": paper["status"] == P.PAT_STATUS_CONVERGED}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        best, gaps = P.pat_tune_step_ratio(geo.handle, f, P.make_params(reg=P.PAT_WAV, alpha=0.02, wavelet_levels=4,
                                                                        wavelet_kind=kind),
                                           [1.0, 3.0, 10.0, 30.0], args.probe_iters, stream)
        e1.record(stream)
        e1.synchronize()
        probe_s = e0.elapsed_time(e1) / 1e3
        tuned = run(args.ttg_max_iters, 1e-4, best)
        out["time_to_gap_tuned"] = {"step_ratio": best, "probe_seconds": probe_s, "iters": tuned["iters_done"],
                                    "seconds": probe_s + tuned["ms"] / 1e3,
                                    "reached": tuned["status"] == P.PAT_STATUS_CONVERGED}
        return out
    return {"dtcwt": leg(P.PAT_WAVELET_DTCWT), "dwt": leg(P.PAT_WAVELET_DWT)}


def run_preprocess(P, S, np, torch, device, stream, geo, w, flush):
    """pat_preprocess on the benchmark geometry: synthetic pressures and calibrations of
    the benchmark's data, timed with CUDA events (mean of 20 calls after 3 warm-ups)."""
    D, T = w["det_xy"].shape[0], w["n_t"]
    rng = np.random.default_rng(7)
    t = w["r0"] + (np.arange(T) + 0.5) * w["dr"]
    f = np.exp(-((t[None, :] - rng.uniform(0.6, 2.0, D)[:, None]) / 0.1) ** 2)
    xp = (0.05, -0.1)
    p, pcal = S.pressure_measurement(f, w["det_xy"], xp, w["r0"], w["dr"], width=2.5 * w["dr"], noise_level=0.01,
                                     seed=0)
    pd = torch.from_numpy(p.astype(np.float32)).to(device)
    cd = torch.from_numpy(pcal.astype(np.float32)).to(device)
    out = torch.empty(D, T, device=device)
    for _ in range(3):
        P.pat_preprocess(geo.handle, pd, cd, xp, 1e-3, out, stream)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        P.pat_preprocess(geo.handle, pd, cd, xp, 1e-3, out, stream)
    e1.record(stream)
    e1.synchronize()
    us = e0.elapsed_time(e1) / 20 * 1e3
    return {"detectors": D, "samples": T, "us_per_call": us, "gb_per_s": 3 * D * T * 4 / (us * 1e-6) / 1e9}


def time_unet_step(P, WS, torch, net, x8, t8, cw, n, stream, steps=10):
    """Tensor-core throughput of the U-Net training step (batch 8, n x n): CUDA events
    around `steps` steps after 3 untimed ones."""
    loss = torch.zeros(1, device=x8.device)
    for _ in range(3):
        P.pat_unet_train_step(net.handle, x8, t8, cw, 8, n, n, 1e-6, loss, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        P.pat_unet_train_step(net.handle, x8, t8, cw, 8, n, n, 1e-6, loss, stream)
    e1.record(stream)
    e1.synchronize()
    step_ms = e0.elapsed_time(e1) / steps
    fwd_fl, step_fl = WS.unet_flops(8, n, n)
    peaks = load_peaks()
    tf = step_fl / (step_ms * 1e-3) / 1e12
    return {"step_ms": step_ms,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": tf / peaks["bf16_tflops"], "flop_per_step": step_fl,
                         "kernels": "k_conv_wgrad_tc (tcgen05, TMEM accumulators, TMA) for every weight gradient; "
                                    "k_conv_fwd_tc for the forward and data-gradient layers with 32-channel multiples "
                                    "and >= 64 channels on one side; k_conv_fwd (mma.sync) for the 8-channel input "
                                    "and output layers and the 32 -> 32 forward",
                         "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)"}}


def run_unet_step_only(args):
    """--unet-step: only the U-Net training-step timing on random bf16 inputs (base 32
    channels, 4 levels, batch 8, 256 x 256), printed as one JSON line."""
    import torch
    import paper_1707_02245_gb300 as P
    from paper_1707_02245_gb300 import build, warmstart as WS
    build.build()
    P.load()
    device = torch.device("cuda:0")
    stream = torch.cuda.current_stream(device)
    n = 256
    g = torch.Generator(device="cpu").manual_seed(0)
    x8 = torch.randn(8, n, n, 8, generator=g).to(torch.bfloat16).to(device)
    t8 = torch.randn(8, n, n, 8, generator=g).to(device)
    net = WS.UNet(base_ch=32, levels=4, seed=1)
    out = time_unet_step(P, WS, torch, net, x8, t8, [1.0] * 8, n, stream, steps=args.unet_step)
    out["nn_wait_timeouts"] = P.pat_nn_wait_timeouts()
    print(json.dumps({"unet_step": out}))
    return 0


def run_warm_start(P, S, np, torch, device, stream, args):
    """The learned warm start on TGV^2 256^2 vessel problems with 128 detectors: training
    pairs from PDHG (the tuned balance s, rel gap 1e-5, at most --warm-label-iters), U-Net
    training on the GPU, then cold and warm PDHG to rel gap 1e-4 on held-out seeds (one
    lockstep batch each, the same s).  Warm time includes the features, the network and
    the state map."""
    from paper_1707_02245_gb300 import warmstart as WS
    n, ndet, nt = 256, 128, 512
    ws = [S.workload_warm(s, n=n, n_det=ndet, n_t=nt) for s in range(args.warm_train)]
    wv = [S.workload_warm(100000 + s, n=n, n_det=ndet, n_t=nt) for s in range(args.warm_val)]
    w0 = ws[0]
    geo = P.Geometry(n, w0["det_xy"], w0["n_t"], w0["r0"], w0["dr"], w0["quad_m"])
    out = {"workload": f"TGV^2 {n}x{n} vessel phantoms, {ndet} detectors x {nt} samples, noise U[1%,10%], "
                       f"alpha 0.02 beta 0.04", "train_pairs": len(ws), "held_out": len(wv)}
    f0 = WS.simulate(torch, w0, device, stream)
    sr, _ = P.pat_tune_step_ratio(geo.handle, f0, P.make_params(reg=1, alpha=w0["alpha"], beta=w0["beta"]),
                                  [1.0, 3.0, 10.0, 30.0], args.probe_iters, stream)
    out["step_ratio"] = sr
    t0 = time.perf_counter()
    F, T, _, infos = WS.make_pairs(torch, ws, geo, device, stream, iters=args.warm_label_iters, tol=1e-5, batch=64,
                                   step_ratio=sr)
    torch.cuda.synchronize(device)
    its = [i["iters_done"] for i in infos]
    out["labels"] = {"seconds": time.perf_counter() - t0, "iters_median": float(np.median(its)),
                     "converged_1e-5": sum(i["status"] == P.PAT_STATUS_CONVERGED for i in infos)}
    Fv, Tv, fv, _ = WS.make_pairs(torch, wv, geo, device, stream, iters=1, tol=0.0, batch=64, step_ratio=sr)
    e = (T ** 2).mean(dim=(0, 1, 2)).cpu().numpy()
    cw = list((1.0 / np.maximum(e, 1e-12) / len(e)).astype(float))
    net = WS.UNet(base_ch=32, levels=4, seed=1)
    lg, tt = WS.train(torch, net, F, T, args.warm_steps, 8, 1e-3, cw, stream, log_every=max(1, args.warm_steps // 4))
    out["training"] = {"steps": args.warm_steps, "batch": 8, "seconds": tt, "loss_log": lg, "params": net.num_params}
    out["training"].update(time_unet_step(P, WS, torch, net, F[:8].contiguous(), T[:8].contiguous(), cw, n, stream))
    prms = [P.make_params(reg=1, alpha=w["alpha"], beta=w["beta"]) for w in wv]
    # cold
    ci, us_c, ct = WS.solve(torch, geo, fv, wv, device, stream, tol=1e-4, max_iters=30000, step_ratio=sr)
    # warm: features (already computed in Fv) are part of the warm path, so time them again
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    feats = torch.empty_like(Fv)
    for k in range(len(wv)):
        P.pat_warm_start_features(geo.handle, fv[k], feats[k], 8, stream)
    x0s, y0s = WS.predict_states(torch, net, geo, feats, fv, prms, device, stream)
    e1.record(stream)
    e1.synchronize()
    pred_s = e0.elapsed_time(e1) / 1e3
    wi, us_w, wt = WS.solve(torch, geo, fv, wv, device, stream, tol=1e-4, max_iters=30000, x0s=x0s, y0s=y0s,
                            step_ratio=sr)
    cit = np.array([i["iters_done"] for i in ci], dtype=float)
    wit = np.array([i["iters_done"] for i in wi], dtype=float)
    diff = [float((us_c[k] - us_w[k]).norm() / us_c[k].norm()) for k in range(len(wv))]
    out["cold"] = {"iters_median": float(np.median(cit)), "iters_mean": float(cit.mean()), "seconds": ct,
                   "converged": sum(i["status"] == P.PAT_STATUS_CONVERGED for i in ci)}
    out["warm"] = {"iters_median": float(np.median(wit)), "iters_mean": float(wit.mean()), "solve_seconds": wt,
                   "predict_seconds": pred_s, "seconds": wt + pred_s,
                   "converged": sum(i["status"] == P.PAT_STATUS_CONVERGED for i in wi)}
    out["speedup_warm_vs_cold"] = ct / (wt + pred_s)
    out["iters_ratio_median"] = float(np.median(wit / cit))
    out["image_rel_diff_warm_vs_cold_median"] = float(np.median(diff))
    net.close()
    geo.close()
    return out


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "bf16_tflops": float(pk["bf16_tflops"]),
                "sm_max_mhz": float(pk.get("sm_max_mhz", 2070.0)),
                "source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback (profiling recipe)"}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", default="tgv256")
    ap.add_argument("--cpu-iters", type=int, default=2, help="oracle iterations of the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttg", action="store_true")
    ap.add_argument("--ttg-max-iters", type=int, default=60000)
    ap.add_argument("--iters", type=int, default=0,
                    help="override the PDHG iterations per step (short runs for the ncu launch list)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=16, help="TGV 256^2 problems in the lockstep batch (0: skip)")
    ap.add_argument("--mixed", type=int, default=1, help="run the 64-problem mixed batch (0: skip)")
    ap.add_argument("--wavelet-batch", type=int, default=8,
                    help="problems of the wavelet leg's lockstep batch (0 or 1: skip)")
    ap.add_argument("--mixed-max-iters", type=int, default=5000)
    ap.add_argument("--probe-iters", type=int, default=300, help="iterations of each step-ratio probe")
    ap.add_argument("--warm", type=int, default=1, help="run the learned warm-start leg (0: skip)")
    ap.add_argument("--unet-step", type=int, default=0,
                    help="only time this many U-Net training steps (batch 8, 256^2) and print them (0: full run)")
    ap.add_argument("--warm-train", type=int, default=128)
    ap.add_argument("--warm-val", type=int, default=16)
    ap.add_argument("--warm-steps", type=int, default=2000)
    ap.add_argument("--warm-label-iters", type=int, default=10000, help="iteration cap of the training labels")
    ap.add_argument("--no-prep", action="store_true")
    ap.add_argument("--no-wavelet", action="store_true")
    ap.add_argument("--no-update-hbm", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shapes (no autotuner)")
    ap.add_argument("--shape-cache", default="",
                    help="the autotuner's JSON cache (default: a fresh temporary file); shapes found in it are "
                         "applied without timing")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.unet_step:
        return run_unet_step_only(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
