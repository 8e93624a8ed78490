#!/usr/bin/env python3
"""Benchmark of the coupled flood-pedestrian step on B300.

Workload (default): the synthetic shopping centre, 512 x 512 cells of 0.5 m,
10,000 evacuees, evacuee roughness coupling on, triangular depth hydrograph
peaking at 1.0 m.  The simulation is first advanced 1024 steps (flood inside,
evacuation under way) and that state is kept as a snapshot.  One benchmark
step = restore the snapshot (untimed), flush L2, then 256 coupled simulation
steps through the C ABI (``fp_step``), timed with CUDA events on the
simulation's stream.

metric  coupled cell-updates/s + ped-updates/s (cells x steps + pedestrians
        advanced, over the timed region).
e2e     the same through the C ABI with host buffers: pinned-host state and
        pedestrian upload, 256 steps, read-back of h, hu, hv, pedestrians and
        counters, all inside the timed region.
roofline the flood kernel (HBM-bound stencil), 34 algorithmic bytes per cell
        update of the tiles it computed (it skips tiles that stay dry), its
        launch duration from CUDA events in a profiled pass.
cpu_baseline the FP64 C oracle on a bounded sample of the same workload.

``--impl reference`` times the oracle itself (host cores) on the same workload.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling).
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHUNK = 256            # simulation steps per benchmark step
PRE_STEPS = 1024       # steps before the snapshot
FLOOD_BYTES_PER_CELL = 34  # read h,hu,hv,z,n0 (20 B) + occupancy (2 B); write h,hu,hv (12 B)
METRIC = "coupled cell-updates/s + ped-updates/s"
UNIT = "updates/s"


def workload(seed):
    import scenarios
    return scenarios.shopping_centre(512, 0.5, 10_000, 0, seed, 1800.0)


def launches_per_chunk(sc, hash_ahead):
    """Kernel launches of one benchmark step (CHUNK coupled steps after a
    restore): the first step opens with a hashing pass over all records
    (hash_count, flood, scan, gather, pedestrian update: 5 launches); with the
    records hashed ahead and no barrier to build, every later step is the
    flood, scan, gather and pedestrian kernels alone (4), else 5."""
    opening = (not hash_ahead) or (len(sc.barrier_cells) > 0 and sc.n_layers > 0)
    return 5 + (CHUNK - 1) * (5 if opening else 4)


def combine_ranks(t_sec, updates, device):
    """Whole-job figures of independent replicas: the slowest rank's timed
    seconds (MAX) and the updates of all ranks (SUM), over the default process
    group (NCCL on GPUs; gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_sec)], dtype=torch.float64, device=device)
    uu = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


def scenarios_mod():
    import scenarios
    return scenarios


def wet2048():
    """2048 x 2048 cells of 0.5 m holding water almost everywhere (70 % wet,
    velocities up to 1.5 m/s, uneven bed, every boundary type): the flood
    kernel on its full HLL path, as in a flooded shopping centre."""
    return scenarios_mod().random_wet_state(2048, 2048, dx=0.5, seed=5)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes per flood-kernel launch from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum; profiles/flood_kernel_traffic.md), valid only for the
# kernel sources they were taken on.
FLOOD_TRAFFIC = {"sources_sha256": "028ecc7b75e77bf0790eaa4ca4ae2bb0da2c316059374eb0e4a48152c3d8ce79",
                 "shopping_centre_512": 4.52e6, "wet_2048": 93.01e6 + 15.92e6}
FLOOD_SOURCES = ("flood.cu", "flood_dev.cuh", "fp_common.cuh")


def flood_traffic(workload_name):
    """Measured DRAM bytes per launch of the flood kernel on a workload; None
    once the kernel's sources differ from those the counters were taken on."""
    h = hashlib.sha256()
    for f in FLOOD_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1908_05232_b300", "csrc", f), "rb").read())
    if h.hexdigest() != FLOOD_TRAFFIC["sources_sha256"]:
        return None
    return FLOOD_TRAFFIC.get(workload_name)


# --------------------------------------------------------------------------
# oracle (CPU) timing
# --------------------------------------------------------------------------
def oracle_rate(n_steps, seed=2):
    import oracle
    sc = workload(seed)
    o = oracle.Oracle(sc)
    t0 = time.perf_counter()
    upd = 0
    for _ in range(n_steps):
        active = int((o.pexit == 0).sum())
        if o.step_dt() == 0:
            break
        upd += sc.n_cells + active
    el = time.perf_counter() - t0
    return upd / el, el


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    sc = workload(2)
    o = oracle.Oracle(sc)
    per = args.ref_sample_steps
    for _ in range(args.warmup):
        o.step(per)
    t_total, upd = 0.0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per):
            active = int((o.pexit == 0).sum())
            if o.step_dt() == 0:
                break
            upd += sc.n_cells + active
        t_total += time.perf_counter() - t0
    value = upd / t_total
    sample = "%d oracle steps per benchmark step of the 512x512 / 10k-evacuee shopping centre" % per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "shopping_centre_512", "nx": 512, "ny": 512, "dx": 0.5, "n_peds": 10000},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1908_05232_b300 as P
    from paper_1908_05232_b300 import _native as N
    P.build.build()
    sc = workload(2 + rank)
    stream = torch.cuda.Stream()
    sim = P.from_scenario(sc, tile_rows=args.tile_rows)
    N.fp_set_stream(sim.h, stream.cuda_stream)
    sim.step(PRE_STEPS)
    sim.synchronize()
    # device snapshot
    dev = torch.device("cuda", local)
    snap = [torch.empty((sc.ny, sc.nx), dtype=torch.float32, device=dev) for _ in range(3)]
    for k, t in zip((N.FP_FIELD_H, N.FP_FIELD_HU, N.FP_FIELD_HV), snap):
        N.fp_read_state(sim.h, k, t)
    c0 = sim.counters()
    peds_all = sim.peds()
    active = peds_all[peds_all["exited"] == 0].copy()
    peds_dev = torch.from_numpy(active.view(np.uint8).copy()).to(dev)
    n_act = int(active.shape[0])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2

    def restore():
        N.fp_set_state(sim.h, snap[0], snap[1], snap[2])
        N.fp_clear_pedestrians(sim.h)
        N._check(N.lib().fp_add_pedestrians(sim.h, N._VP(peds_dev.data_ptr()), n_act), sim.h)
        sim.n_total = n_act
        N.fp_set_time(sim.h, c0["t_ticks"], c0["step"])
        sim.counters()  # runs the post-restore preparation outside the timed region
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()

    def one(timed):
        restore()
        a = sim.counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(CHUNK)
        e1.record(stream)
        e1.synchronize()
        b = sim.counters()
        if b["error_flags"]:
            raise RuntimeError("device error flags %#x" % b["error_flags"])
        upd = (b["step"] - a["step"]) * sc.n_cells + (b["ped_updates"] - a["ped_updates"])
        return e0.elapsed_time(e1), upd, b["step"] - a["step"]

    # launch shape: the autotuner's candidates timed on this snapshot (the
    # results never depend on the shape); --tile-rows pins the flood tile height
    tuned = {"tile_rows": args.tile_rows or 16, "ped_lanes": 8, "hash_ahead": True}
    if not args.no_tune:
        best = None
        for tr in ((args.tile_rows,) if args.tile_rows else (8, 16, 32)):
            for pl in (4, 8, 16):
                for ha in (True, False):
                    N.fp_set_tuning(sim.h, tr, pl)
                    N.fp_set_hash_ahead(sim.h, ha)
                    t = min(one(False)[0] for _ in range(2))
                    if best is None or t < best[0]:
                        best = (t, tr, pl, ha)
        tuned = {"tile_rows": best[1], "ped_lanes": best[2], "hash_ahead": best[3]}
    N.fp_set_tuning(sim.h, tuned["tile_rows"], tuned["ped_lanes"])
    N.fp_set_hash_ahead(sim.h, tuned["hash_ahead"])

    for _ in range(args.warmup):
        one(False)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ms_list, upd_total, steps_total = [], 0, 0
    for _ in range(args.steps):
        ms, upd, st = one(True)
        ms_list.append(ms)
        upd_total += upd
        steps_total += st
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_sec = sum(ms_list) / 1e3
    if ws > 1:
        t_sec, upd_all = combine_ranks(t_sec, upd_total, dev)
    else:
        upd_all = float(upd_total)
    value = upd_all / t_sec

    # profiled pass: CUDA events around each kernel group, same workload
    restore()
    N.fp_set_profiling(sim.h, 1)
    sim.step(CHUNK)
    prof = sim.profile()
    N.fp_set_profiling(sim.h, 0)
    flood_ms = prof["flood_ms"] / max(prof["steps"], 1)
    hbm, peak_kind = peaks()
    # algorithmic bytes: the cells of the tiles the kernel computed (dry tiles
    # it skips move no bytes)
    flood_cells = prof["flood_cells"] / max(prof["steps"], 1)
    achieved = flood_cells * FLOOD_BYTES_PER_CELL / (flood_ms * 1e-3) / 1e9
    traffic = flood_traffic("shopping_centre_512")

    # end to end through the C ABI with pinned host buffers
    host_state = [t.cpu().pin_memory() for t in snap]
    host_peds = torch.from_numpy(active.view(np.uint8).copy()).pin_memory()
    out_state = [torch.empty((sc.ny, sc.nx), dtype=torch.float32).pin_memory() for _ in range(3)]
    out_peds = torch.empty(n_act * 32, dtype=torch.uint8).pin_memory()
    e2e_t = 0.0
    for it in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        N.fp_set_state(sim.h, host_state[0], host_state[1], host_state[2])
        N.fp_clear_pedestrians(sim.h)
        N._check(N.lib().fp_add_pedestrians(sim.h, N._VP(host_peds.data_ptr()), n_act), sim.h)
        sim.n_total = n_act
        N.fp_set_time(sim.h, c0["t_ticks"], c0["step"])
        sim.step(CHUNK)
        for k, t in zip((N.FP_FIELD_H, N.FP_FIELD_HU, N.FP_FIELD_HV), out_state):
            N.fp_read_state(sim.h, k, t)
        N._check(N.lib().fp_read_state(sim.h, N.FP_FIELD_PEDS, N._VP(out_peds.data_ptr()), n_act * 32), sim.h)
        sim.counters()
        el = time.perf_counter() - t0
        if it >= args.warmup:
            e2e_t += el
    # every iteration replays the same 256 steps from the snapshot (deterministic),
    # so it performs the same updates as a device-timed iteration
    e2e_value = (upd_total / args.steps) * args.steps / e2e_t
    h2d = 3 * sc.n_cells * 4 + n_act * 32
    d2h = 3 * sc.n_cells * 4 + n_act * 32 + ctypes.sizeof(N.FpCounters)

    # the same kernel where it is HBM-bound: a 2048x2048 grid holding water
    # almost everywhere (no pedestrians, so the kernel runs alone), CUDA events
    # around the flood kernel in a profiled pass
    roof2048 = None
    if rank == 0 and not args.no_2048:
        big = wet2048()
        bsim = P.from_scenario(big, peds=False)
        N.fp_set_stream(bsim.h, stream.cuda_stream)
        bsim.step(4)
        bsim.synchronize()
        N.fp_set_profiling(bsim.h, 1)
        bsim.step(32)
        bprof = bsim.profile()
        N.fp_set_profiling(bsim.h, 0)
        bflood = bprof["flood_ms"] / max(bprof["steps"], 1)
        bcells = bprof["flood_cells"] / max(bprof["steps"], 1)
        bach = bcells * FLOOD_BYTES_PER_CELL / (bflood * 1e-3) / 1e9
        roof2048 = {"kernel": "flood_kernel<16>", "workload": "wet_2048 (2048x2048 cells of 0.5 m, 70 % wet, every boundary type)",
                    "bound": "hbm", "achieved": bach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": bach / hbm, "us_per_launch": bflood * 1e3, "bytes_per_cell_update": FLOOD_BYTES_PER_CELL,
                    "computed_cells_per_launch": bcells,
                    "traffic": flood_traffic("wet_2048"), "note": "profiled pass, no pedestrians: the kernel timed alone"}
        bsim.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, el = oracle_rate(args.cpu_sample_steps)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "first %d coupled steps of the same 512x512 / 10k-evacuee workload, FP64 C oracle, "
                         "single thread (%.1f s)" % (args.cpu_sample_steps, el)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms_list), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "shopping_centre_512", "nx": sc.nx, "ny": sc.ny, "dx": sc.dx,
                       "n_peds": sc.n_peds, "n_peds_active_at_snapshot": n_act,
                       "sim_steps_per_bench_step": CHUNK, "snapshot_after_steps": PRE_STEPS,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed between timed iterations (256 MB write); the 512x512 working set "
                             "(~10 MB) is L2-resident within an iteration",
                       "tile_rows": tuned["tile_rows"], "ped_lanes": tuned["ped_lanes"],
                       "hash_ahead": tuned["hash_ahead"],
                       "launch_shape": "default" if args.no_tune else "fastest autotuner candidate on the snapshot"},
            "breakdown": {"cell_updates_per_s": steps_total * sc.n_cells / (sum(ms_list) / 1e3),
                          "ped_updates_per_s": (upd_total - steps_total * sc.n_cells) / (sum(ms_list) / 1e3),
                          "profiled_ms_per_step": {k: prof[k] / max(prof["steps"], 1)
                                                   for k in ("hash_ms", "flood_ms", "ped_chain_ms", "step_ms")}},
            "roofline": {"kernel": "flood_kernel<%d>" % tuned["tile_rows"], "bound": "hbm", "achieved": achieved,
                         "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                         "bytes_per_cell_update": FLOOD_BYTES_PER_CELL,
                         "computed_cells_per_launch": flood_cells, "cells_per_launch": sc.n_cells,
                         "note": "512x512 fits in L2; frac is against HBM; bytes counted for the cells of "
                                 "the tiles computed (dry tiles are skipped)"},
            "roofline_2048": roof2048,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clocks,
            "gpu_launches": launches_per_chunk(sc, tuned["hash_ahead"]) * args.steps,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_surrogate(args):
    """Learned surrogate against the plain update on the 2048x2048 shopping
    centre with 100,000 coupled pedestrians (500 responders building a 2-layer
    barrier; flood from t = 900 s): two identical simulations are brought to
    mid-flood (CFL step), then the same simulated interval is run with the plain
    update at a fixed 2^-5 s step and with surrogate windows of 8 such steps
    (default guard: per-tile mass bound 1e-4, plain check every 64 steps,
    suspension above 1 cm).  Metric: simulated seconds per wall second;
    accuracy: the largest depth difference between the two runs at the end."""
    import torch
    import scenarios
    import paper_1908_05232_b300 as P
    from paper_1908_05232_b300 import _native as N
    torch.cuda.set_device(0)
    P.build.build()
    dt = 2.0 ** -5
    sc = scenarios.config_barrier()
    t_start = args.surrogate_start
    sur = P.Surrogate.pretrained()
    t0 = time.perf_counter()
    sims = []
    for _ in range(2):
        sim = P.from_scenario(sc)
        c = sim.counters()
        while c["t_ticks"] < int(t_start * N.TICKS):
            sim.step(256)
            c = sim.counters()
        sim.set_fixed_dt(dt)
        sims.append(sim)
    setup = time.perf_counter() - t0
    plain, surr = sims
    assert plain.counters()["t_ticks"] == surr.counters()["t_ticks"]
    windows = args.steps * 8
    # warm-up: one window each (graphs, scratch buffers), on both simulations
    plain.step(8)
    plain.synchronize()
    st_w = surr.surrogate_advance(sur, 1, fix_tol=args.surrogate_fix_tol)
    torch.cuda.synchronize()
    ta = plain.counters()["t_ticks"]
    t0 = time.perf_counter()
    plain.step(8 * windows)
    plain.synchronize()
    t_plain = time.perf_counter() - t0
    tb = plain.counters()["t_ticks"]
    ts0 = surr.counters()["t_ticks"]
    t0 = time.perf_counter()
    st = surr.surrogate_advance(sur, windows, fix_tol=args.surrogate_fix_tol)
    t_sur = time.perf_counter() - t0
    tc = surr.counters()["t_ticks"]
    sim_s = (tb - ta) / N.TICKS
    sim_s_sur = (tc - ts0) / N.TICKS
    err = float(np.abs(plain.field(N.FP_FIELD_H) - surr.field(N.FP_FIELD_H)).max())
    wet_frac = float((plain.field(N.FP_FIELD_H) > 0).mean())
    rate_p, rate_s = sim_s / t_plain, sim_s_sur / t_sur
    line = {"metric": "scenario-seconds/s (learned surrogate windows vs plain update)", "value": rate_s,
            "unit": "scenario-s/s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": 1e3 * t_sur / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 net (FP32 accumulate), f32 plain update", "data": "synthetic",
            "config": {"workload": "surrogate_2048 (2048x2048 shopping centre, 100,000 pedestrians, barrier, "
                                   "flood from 900 s)", "start_s": t_start, "dt_s": dt,
                       "windows": windows, "steps_per_window": 8, "wet_fraction_at_end": wet_frac,
                       "guard": {"mass_tol": 1e-4, "fix_tol": args.surrogate_fix_tol, "check_tol_m": 0.01,
                                 "check_every_windows": 8, "suspend_windows": 8},
                       "setup_s": setup},
            "plain": {"value": rate_p, "unit": "scenario-s/s", "seconds": t_plain},
            "speedup_vs_plain": rate_s / rate_p,
            "max_depth_error_m": err,
            "guard": {k: getattr(st, k) for k, _ in st._fields_}}
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args):
    """Batched ensemble: 256 seeded shopping-centre scenarios (grid side 128-1024,
    1k-50k pedestrians, 50-1000 responders, 1-3 sandbag layers, inflow peak
    0.3-1.5 m) stepped together by the batched kernels, against the same
    simulations stepped one by one.  Metric: simulated scenario-seconds per
    wall second."""
    import torch
    import scenarios
    import paper_1908_05232_b300 as P
    torch.cuda.set_device(0)
    P.build.build()
    scs = scenarios.ensemble(args.ensemble_size)
    t0 = time.perf_counter()
    sims = [P.from_scenario(sc) for sc in scs]
    setup = time.perf_counter() - t0
    batch = P.Batch(sims)
    chunk = 64
    for _ in range(args.warmup):
        batch.step(chunk)
    batch.synchronize()

    def sim_seconds():
        return sum(s.counters()["t_ticks"] for s in sims) / float(1 << 20)

    def cell_steps():
        return sum(s.counters()["step"] * s.nx * s.ny for s in sims)

    s0, c0 = sim_seconds(), cell_steps()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        batch.step(chunk)
    batch.synchronize()
    t_batch = time.perf_counter() - t0
    s1, c1 = sim_seconds(), cell_steps()
    batch.close()
    # the simulations' own step graphs (a step whose records are not yet hashed
    # ahead, then one whose are) captured before the timed arms, as the batch's
    # were in its warm-up
    for sim in sims:
        sim.step(2 * chunk)
        sim.synchronize()
    s1w, c1w = sim_seconds(), cell_steps()
    # one by one: each simulation's steps run to completion before the next starts
    t0 = time.perf_counter()
    for sim in sims:
        sim.step(chunk * args.steps)
        sim.synchronize()
    t_single = time.perf_counter() - t0
    s2, c2 = sim_seconds(), cell_steps()
    # independent: every simulation on its own stream, all enqueued at once
    t0 = time.perf_counter()
    for sim in sims:
        sim.step(chunk * args.steps)
    for sim in sims:
        sim.synchronize()
    t_streams = time.perf_counter() - t0
    s3 = sim_seconds()
    rate_b = (s1 - s0) / t_batch
    rate_1 = (s2 - s1w) / t_single
    rate_s = (s3 - s2) / t_streams
    line = {"metric": "scenario-seconds/s (batched ensemble)", "value": rate_b, "unit": "scenario-s/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ensemble_%d" % len(scs), "scenarios": len(scs),
                       "cells": int(sum(sc.nx * sc.ny for sc in scs)), "pedestrians": int(sum(sc.n_peds for sc in scs)),
                       "sim_steps_per_bench_step": chunk, "setup_s": setup},
            "one_by_one": {"value": rate_1, "unit": "scenario-s/s", "seconds": t_single},
            "independent_streams": {"value": rate_s, "unit": "scenario-s/s", "seconds": t_streams},
            "speedup_vs_one_by_one": rate_b / rate_1,
            "speedup_vs_independent_streams": rate_b / rate_s,
            "cell_updates_per_s_batched": (c1 - c0) / t_batch, "cell_updates_per_s_one_by_one": (c2 - c1w) / t_single}
    print(json.dumps(line), flush=True)
    return 0


def run_case(args):
    """A short run of one workload (the command line profiled under ncu): after
    an optional pre-run to a simulated time, the case's steps in the given
    launch shape, timed with CUDA events on the simulation's stream (a time
    taken under a profiler is not a measurement)."""
    import torch
    import scenarios
    import paper_1908_05232_b300 as P
    torch.cuda.set_device(0)
    P.build.build()
    if args.ncu_case == "barrier2048":
        sc = scenarios.config_barrier()
    elif args.ncu_case == "wet2048":
        sc = wet2048()
    else:
        sc = workload(2)
    from paper_1908_05232_b300 import _native as N
    sim = P.from_scenario(sc, tile_rows=args.tile_rows)
    stream = torch.cuda.Stream()
    N.fp_set_stream(sim.h, stream.cuda_stream)
    N.fp_set_tuning(sim.h, args.tile_rows or 16, args.case_lanes)
    N.fp_set_hash_ahead(sim.h, args.case_hash_ahead != 0)
    if args.case_time > 0:
        # run up to the simulated time first, then open the profiler range
        # (ncu --profile-from-start off) around the case's steps only
        while sim.counters()["t_ticks"] < int(args.case_time * N.TICKS):
            sim.step(256)
        sim.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.case_steps)
    e1.record(stream)
    sim.synchronize()
    if args.case_time > 0:
        torch.cuda.cudart().cudaProfilerStop()
    c = sim.counters()
    print(json.dumps({"case": args.ncu_case, "steps": c["step"], "t_ticks": c["t_ticks"],
                      "n_active": c["n_active"], "error_flags": c["error_flags"],
                      "ped_lanes": args.case_lanes, "hash_ahead": args.case_hash_ahead,
                      "us_per_step": 1e3 * e0.elapsed_time(e1) / max(args.case_steps, 1)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--no-2048", action="store_true", help="skip the 2048x2048 flood-kernel roofline pass")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (16-row tiles, 8 lanes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=100)
    ap.add_argument("--ref-sample-steps", type=int, default=8)
    ap.add_argument("--ncu-case", choices=["barrier2048", "wet2048", "shopping512"], default=None,
                    help="short untimed run of one workload, for profiler captures")
    ap.add_argument("--case-steps", type=int, default=4)
    ap.add_argument("--case-lanes", type=int, default=8, choices=[4, 8, 16], help="lanes per pedestrian in the case")
    ap.add_argument("--case-hash-ahead", type=int, default=1, choices=[0, 1], help="hash-ahead in the case")
    ap.add_argument("--case-time", type=float, default=0.0,
                    help="simulated seconds to run before the case's steps (profiler range opened after them)")
    ap.add_argument("--workload", choices=["shopping512", "ensemble", "surrogate"], default="shopping512")
    ap.add_argument("--surrogate-start", type=float, default=1500.0, help="simulated time (s) the surrogate run starts at")
    ap.add_argument("--surrogate-fix-tol", type=float, default=0.0,
                    help="accept net tiles up to this mass residual and close their balance (0: the 1e-4 bound)")
    ap.add_argument("--ensemble-size", type=int, default=256)
    args = ap.parse_args()
    if args.ncu_case:
        return run_case(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
