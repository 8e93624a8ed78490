#!/usr/bin/env python3
"""Benchmark of the coupled flood-pedestrian step on B300.

Workload (default): the pre-flood barrier deployment at scale taken up
mid-flood -- 2048 x 2048 cells of 0.5 m, 100,000 pedestrians of which 500
responders building a 200-cell, 2-layer sandbag barrier, evacuee roughness
coupling on, the triangular depth hydrograph at its 1.0 m peak (t = 1500 s),
the synthetic mid-flood state of ``scenarios.config_barrier_midflood`` (9 %
of the cells wet, the water within 300 m of the breach, the responders
mid-deployment).  One benchmark step =
restore that snapshot (untimed), flush L2, then 512 coupled simulation steps
through the C ABI (``fp_step``), timed with CUDA events on the simulation's
stream.

metric  coupled cell-updates/s + ped-updates/s (cells x steps + pedestrians
        advanced, over the timed region); ``breakdown`` gives the cell updates
        the flood kernel computed (it skips tiles that stay dry) beside all.
e2e     the same through the C ABI with host buffers: pinned-host state, bed
        and pedestrian upload, 512 steps, read-back of h, hu, hv, pedestrians
        and counters, all inside the timed region.
roofline the flood kernel (HBM-bound stencil), 34 algorithmic bytes per cell
        update of the tiles it computed, its launch duration from CUDA events
        on its own stream in a profiled pass of the same steps;
        ``roofline_peds`` the pedestrian kernel, 96 algorithmic bytes per
        pedestrian update; ``roofline_muscl_wet2048`` the second-order
        update's two stage kernels on the wet grid (74 B per cell and step);
        ``roofline_wet2048`` the flood kernel alone on a
        2048 x 2048 grid holding water almost everywhere.
cpu_baseline the FP64 C oracle on one coupled step of the same snapshot.
batched  a seeded ensemble of shopping centres stepped together (per-step
        batch kernels in graphs, and one persistent launch per 256 steps: the
        faster is ``value``) against the same simulations stepped one by one
        (scenario-seconds/s).
surrogate the learned surrogate's windows against the plain update from the
        same snapshot at a fixed step (scenario-seconds/s), with the largest
        depth difference from the plain run at the end.

Other workloads (``--workload``): ``ensemble`` and ``surrogate`` (the batched
and surrogate figures at full size), ``deployment`` (the Section 3.3 study of
36 runs as one batch), ``scenario1`` (the Section 3.2 study: entry/exit flow
through the doors, flood, evacuation, with and without the roughness coupling).

``--impl reference`` times the oracle itself (host cores) on the same snapshot.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling).
"""
import argparse
import ctypes
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHUNK = 512            # simulation steps per benchmark step
FLOOD_BYTES_PER_CELL = 34  # read h,hu,hv,z,n0 (20 B) + occupancy (2 B); write h,hu,hv (12 B)
# second order, per cell and step: stage 1 reads h,hu,hv,z (16 B) and writes the
# stage state (12 B); stage 2 reads it (12 B), z, n0 (8 B), the occupancy (2 B)
# and the step's start state (12 B) and writes h,hu,hv (12 B)
MUSCL_BYTES_PER_CELL = 74
# pedestrian update: read its record (32 B) and position copy (8 B), its cell's
# h, hu, hv (12 B), navigation code, arrival and cell flags (3 B); write its
# record (32 B), hash key and slot (8 B), its evacuee count (1 B amortised)
PED_BYTES = 96
METRIC = "coupled cell-updates/s + ped-updates/s"
UNIT = "updates/s"
WORKLOAD = "barrier_2048_midflood"
WORKLOAD_TEXT = ("2048x2048 cells of 0.5 m, 100,000 pedestrians (500 responders, 200-cell 2-layer sandbag "
                 "barrier), synthetic mid-flood state at t = 1500 s")


def workload(seed):
    import scenarios
    return scenarios.config_barrier_midflood(seed)


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


def host_cpu():
    model = platform.processor() or "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model}


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


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per flood-kernel
# launch from ncu captures of the kernel sources with this hash: the mid-flood
# barrier case in the benchmark's tuned shape (8-row runs) and the wet grid
# (16-row runs)
FLOOD_TRAFFIC = {"sources_sha256": "ea3c758bdcb0678f4701bed21628187c6212c4ad10392e72562a7157ca119d49",
                 "barrier_2048_midflood": 21734784, "wet_2048": 115072256}
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
def oracle_steps(o, sc, n_steps, budget_s=None):
    """Coupled oracle steps; returns (updates, seconds, steps taken), stopping
    early once budget_s seconds have been spent."""
    t_total, upd, k = 0.0, 0, 0
    for _ in range(n_steps):
        active = int(o.counters()["n_active"])
        t0 = time.perf_counter()
        dt = o.step_dt()
        t_total += time.perf_counter() - t0
        if dt == 0:
            break
        upd += sc.n_cells + active
        k += 1
        if budget_s is not None and t_total >= budget_s:
            break
    return upd, t_total, k


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    sc = workload(3)
    o = oracle.Oracle(sc)
    # one oracle coupled step stands for one benchmark step of the GPU arm (a
    # bounded sample of its 512); warm-up is one untimed step, and the timed
    # steps stop once the budget is spent
    for _ in range(min(args.warmup, 1)):
        o.step(1)
    upd, t_total, k = oracle_steps(o, sc, args.steps, budget_s=args.ref_budget_s)
    value = upd / t_total
    cpu = host_cpu()
    sample = ("%d coupled oracle steps (FP64 C, single thread, %.1f s) of the %s snapshot, after %d untimed; "
              "each stands for one %d-step benchmark step; host %s, %d cores"
              % (k, t_total, WORKLOAD, min(args.warmup, 1), CHUNK, cpu["model"], cpu["nproc"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": k, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * t_total / max(k, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_TEXT, "nx": sc.nx, "ny": sc.ny, "dx": sc.dx,
                       "n_peds": sc.n_peds, "t0_s": sc.t0_ticks / float(1 << 20)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "nproc": cpu["nproc"], "cpu_model": cpu["model"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
class Snapshot:
    """A simulation's start state kept on the device and restored through the
    C ABI before every benchmark step (untimed)."""

    def __init__(self, P, N, sim, sc, dev):
        import torch
        self.N, self.sim, self.sc = N, sim, sc
        c = np.ascontiguousarray
        self.fields = [torch.from_numpy(c(a, np.float32)).to(dev) for a in (sc.h, sc.hu, sc.hv, sc.z)]
        recs = P.ped_records(sc.peds)
        self.n_peds = int(recs.shape[0])
        self.peds = torch.from_numpy(recs.view(np.uint8).copy()).to(dev)

    def restore(self, fields=None, peds=None):
        N, h = self.N, self.sim.h
        f = self.fields if fields is None else fields
        p = self.peds if peds is None else peds
        N.fp_set_state(h, f[0], f[1], f[2])
        N.fp_set_bed(h, f[3])
        N.fp_clear_pedestrians(h)
        N._check(N.lib().fp_add_pedestrians(h, N._VP(p.data_ptr()), self.n_peds), h)
        N.fp_set_time(h, self.sc.t0_ticks, self.sc.step0)
        N.fp_set_barrier_progress(h, self.sc.bags0, self.sc.applied0)


def batched_figures(P, args, dev):
    """A seeded ensemble of shopping centres (grid side 128-1024, 1k-50k
    pedestrians, 50-1000 responders, 1-3 sandbag layers, inflow peak 0.3-1.5
    m) stepped together -- by the per-step batch kernels (64-step graphs, the
    members' launch shapes autotuned on a scratch batch) and by one persistent
    launch per 256 steps -- against the same simulations stepped one by one in
    the default shape, each arm warmed (graphs captured) before its timing."""
    import torch
    import scenarios
    from paper_1908_05232_b300 import autotune
    t0 = time.perf_counter()
    scs = scenarios.ensemble(args.ensemble_size)
    # members' launch shapes tuned on a scratch batch of the same scenarios
    tuned = autotune.tune_batch(scs)
    t_tune = time.perf_counter() - t0
    sims = [P.from_scenario(sc) for sc in scs]
    autotune.apply_batch(sims, tuned["shapes"])
    setup = time.perf_counter() - t0 - t_tune
    chunk, reps = 64, args.ensemble_steps

    def sim_seconds():
        return sum(s.counters()["t_ticks"] for s in sims) / float(1 << 20)

    batch = P.Batch(sims)
    batch.step(chunk)
    batch.synchronize()
    s0 = sim_seconds()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        batch.step(chunk)
    batch.synchronize()
    t_batch = time.perf_counter() - t0
    s1 = sim_seconds()
    # the same ensemble in one persistent launch per 256 steps
    from paper_1908_05232_b300 import _native as N
    t_pers = None
    if N.lib().fp_batch_set_step_mode(batch.h, N.FP_MODE_PERSISTENT) == N.FP_OK:
        batch.step(chunk)
        batch.synchronize()
        sp0 = sim_seconds()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.step(chunk * reps)
        batch.synchronize()
        t_pers = time.perf_counter() - t0
        sp1 = sim_seconds()
    batch.close()
    autotune.apply_batch(sims, [(16, 8)] * len(sims))  # one by one: the default shape
    for sim in sims:  # the members' own step graphs (hashing and hashed-ahead openings)
        sim.step(2 * chunk)
        sim.synchronize()
    s1w = sim_seconds()
    t0 = time.perf_counter()
    for sim in sims:
        sim.step(chunk * reps)
        sim.synchronize()
    t_single = time.perf_counter() - t0
    s2 = sim_seconds()
    for sim in sims:
        sim.close()
    rate_b, rate_1 = (s1 - s0) / t_batch, (s2 - s1w) / t_single
    rate_p = (sp1 - sp0) / t_pers if t_pers else None
    best = max(rate_b, rate_p or 0.0)
    return {"value": best, "unit": "scenario-s/s", "one_by_one": rate_1, "speedup_vs_one_by_one": best / rate_1,
            "kernels_graphs": rate_b, "persistent": rate_p,
            "mode": "persistent" if rate_p and rate_p > rate_b else "kernels_graphs",
            "scenarios": len(scs), "cells": int(sum(sc.nx * sc.ny for sc in scs)),
            "pedestrians": int(sum(sc.n_peds for sc in scs)), "steps_timed": chunk * reps,
            "seconds": {"batched": t_batch, "persistent": t_pers, "one_by_one": t_single, "setup": setup,
                        "tuning": t_tune},
            "tuned_shapes": {"%dx%d" % sh: tuned["shapes"].count(sh) for sh in sorted(set(tuned["shapes"]))},
            "uniform_shape_us_per_step": tuned["uniform"],
            "workload": "ensemble(%d): shopping centres of side 128-1024 cells (0.5 m), 1k-50k pedestrians"
                        % len(scs)}


def surrogate_figures(P, N, sc, args):
    """The learned surrogate's windows (8 fixed steps of 2^-5 s each, default
    guard) against the plain update, both from the benchmark snapshot."""
    import torch
    dt = 2.0 ** -5
    sur = P.Surrogate.pretrained()
    sims = [P.from_scenario(sc) for _ in range(2)]
    for s in sims:
        s.set_fixed_dt(dt)
    plain, surr = sims
    windows = args.surrogate_windows
    plain.step(8)
    plain.synchronize()
    surr.surrogate_advance(sur, 1)
    torch.cuda.synchronize()
    ta = plain.counters()["t_ticks"]
    t0 = time.perf_counter()
    plain.step(8 * windows)
    plain.synchronize()
    t_plain = time.perf_counter() - t0
    tb = plain.counters()["t_ticks"]
    ts0 = surr.counters()["t_ticks"]
    t0 = time.perf_counter()
    st = surr.surrogate_advance(sur, windows)
    t_sur = time.perf_counter() - t0
    tc = surr.counters()["t_ticks"]
    hp, hs = plain.field(N.FP_FIELD_H), surr.field(N.FP_FIELD_H)
    err = float(np.abs(hp - hs).max())
    rate_p, rate_s = (tb - ta) / N.TICKS / t_plain, (tc - ts0) / N.TICKS / t_sur
    out = {"value": rate_s, "unit": "scenario-s/s", "plain": rate_p, "speedup_vs_plain": rate_s / rate_p,
           "max_depth_error_m": err, "meets_1cm": err <= 0.01, "windows": windows, "dt_s": dt,
           "seconds": {"surrogate": t_sur, "plain": t_plain},
           "guard": {k: getattr(st, k) for k, _ in st._fields_}}
    for s in sims:
        s.close()
    sur.close()
    return out


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
    sc = workload(3 + rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    sim = P.from_scenario(sc, tile_rows=args.tile_rows)
    N.fp_set_stream(sim.h, stream.cuda_stream)
    snap = Snapshot(P, N, sim, sc, dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2

    def restore():
        snap.restore()
        sim.counters()  # runs the post-restore preparation outside the timed region
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()

    def one():
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
        st = b["step"] - a["step"]
        upd = st * sc.n_cells + (b["ped_updates"] - a["ped_updates"])
        return e0.elapsed_time(e1), upd, st, b["ped_updates"] - a["ped_updates"]

    # launch shape: the autotuner's candidates timed on this snapshot (the
    # results never depend on the shape); --tile-rows pins the flood tile height
    tuned = {"tile_rows": args.tile_rows or 16, "ped_lanes": 8, "hash_ahead": True}
    if not args.no_tune:
        best = None
        for tr in ((args.tile_rows,) if args.tile_rows else (8, 16, 32)):
            for pl in (1, 2, 4, 8, 16):
                for ha in (True, False):
                    N.fp_set_tuning(sim.h, tr, pl)
                    N.fp_set_hash_ahead(sim.h, ha)
                    t = min(one()[0] for _ in range(2))
                    if best is None or t < best[0]:
                        best = (t, tr, pl, ha)
        tuned = {"tile_rows": best[1], "ped_lanes": best[2], "hash_ahead": best[3]}
    N.fp_set_tuning(sim.h, tuned["tile_rows"], tuned["ped_lanes"])
    N.fp_set_hash_ahead(sim.h, tuned["hash_ahead"])

    for _ in range(args.warmup):
        one()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ms_list, upd_total, steps_total, ped_total = [], 0, 0, 0
    for _ in range(args.steps):
        ms, upd, st, pu = one()
        ms_list.append(ms)
        upd_total += upd
        steps_total += st
        ped_total += pu
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_sec = sum(ms_list) / 1e3
    if ws > 1:
        t_sec, upd_all = combine_ranks(t_sec, upd_total, dev)
    else:
        upd_all = float(upd_total)
    value = upd_all / t_sec
    ms_step = statistics.mean(ms_list)

    # profiled pass: the same steps captured with CUDA events between the
    # kernels (on the stream each kernel runs on) and replayed
    restore()
    N.fp_set_profiling(sim.h, 1)
    sim.step(CHUNK)
    prof = sim.profile()
    N.fp_set_profiling(sim.h, 0)
    nprof = max(prof["steps"], 1)
    flood_ms = prof["flood_ms"] / nprof
    ped_ms = prof["ped_ms"] / nprof
    hbm, peak_kind = peaks()
    flood_cells = prof["flood_cells"] / nprof  # cells of the tiles computed (dry tiles are skipped)
    achieved = flood_cells * FLOOD_BYTES_PER_CELL / (flood_ms * 1e-3) / 1e9
    peds_per_step = ped_total / max(steps_total, 1)
    ped_achieved = peds_per_step * PED_BYTES / (ped_ms * 1e-3) / 1e9 if ped_ms > 0 else None

    # end to end through the C ABI with pinned host buffers
    host_fields = [t.cpu().pin_memory() for t in snap.fields]
    host_peds = snap.peds.cpu().pin_memory()
    n_act = snap.n_peds
    out_state = [torch.empty((sc.ny, sc.nx), dtype=torch.float32).pin_memory() for _ in range(3)]
    out_peds = torch.empty(n_act * 32, dtype=torch.uint8).pin_memory()
    e2e_t, e2e_upd = 0.0, 0
    for it in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        snap.restore(host_fields, host_peds)
        a = sim.counters()
        sim.step(CHUNK)
        for k, t in zip((N.FP_FIELD_H, N.FP_FIELD_HU, N.FP_FIELD_HV), out_state):
            N.fp_read_state(sim.h, k, t)
        N._check(N.lib().fp_read_state(sim.h, N.FP_FIELD_PEDS, N._VP(out_peds.data_ptr()), n_act * 32), sim.h)
        b = sim.counters()
        el = time.perf_counter() - t0
        if it >= args.warmup:
            e2e_t += el
            e2e_upd += (b["step"] - a["step"]) * sc.n_cells + (b["ped_updates"] - a["ped_updates"])
    e2e_value = e2e_upd / e2e_t
    h2d = 4 * sc.n_cells * 4 + n_act * 32
    d2h = 3 * sc.n_cells * 4 + n_act * 32 + 2 * ctypes.sizeof(N.FpCounters)

    # the same kernel where it is HBM-bound: a 2048x2048 grid holding water
    # almost everywhere (no pedestrians, so the kernel runs alone)
    roof_wet = roof_muscl = None
    if rank == 0 and not args.no_wet2048:
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
        roof_wet = {"kernel": "flood_kernel<16>", "workload": "wet_2048 (2048x2048 cells of 0.5 m, 70 % wet, "
                    "every boundary type)", "bound": "hbm", "achieved": bach, "peak": hbm, "peak_kind": peak_kind,
                    "unit": "GB/s", "frac": bach / hbm, "us_per_launch": bflood * 1e3,
                    "bytes_per_cell_update": FLOOD_BYTES_PER_CELL, "computed_cells_per_launch": bcells,
                    "traffic": flood_traffic("wet_2048"), "note": "profiled pass, no pedestrians: the kernel alone"}
        bsim.close()
        # the second-order update (the cited scheme at full order) on the same grid
        big.order = 2
        msim = P.from_scenario(big, peds=False)
        N.fp_set_stream(msim.h, stream.cuda_stream)
        msim.step(4)
        msim.synchronize()
        N.fp_set_profiling(msim.h, 1)
        msim.step(32)
        mprof = msim.profile()
        N.fp_set_profiling(msim.h, 0)
        mflood = mprof["flood_ms"] / max(mprof["steps"], 1)
        mach = big.n_cells * MUSCL_BYTES_PER_CELL / (mflood * 1e-3) / 1e9
        roof_muscl = {"kernel": "muscl_stage_kernel<1>+<2>", "workload": "wet_2048, fp_config.order = 2",
                      "bound": "hbm", "achieved": mach, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                      "frac": mach / hbm, "us_per_step": mflood * 1e3, "bytes_per_cell_step": MUSCL_BYTES_PER_CELL,
                      "cells_per_step": big.n_cells, "traffic": None,
                      "note": "profiled pass, no pedestrians: the two stage kernels of a step, every cell computed"}
        msim.close()

    sim.close()
    batched = surrogate = None
    if rank == 0 and not args.no_batched:
        batched = batched_figures(P, args, dev)
    if rank == 0 and not args.no_surrogate:
        surrogate = surrogate_figures(P, N, sc, args)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        o = oracle.Oracle(sc)
        upd, el, k = oracle_steps(o, sc, args.cpu_sample_steps)
        hc = host_cpu()
        cpu = {"value": upd / el, "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": hc["nproc"],
               "cpu_model": hc["model"],
               "sample": "%d coupled step(s) of the same %s snapshot, FP64 C oracle, single thread (%.1f s)"
                         % (k, WORKLOAD, el)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "description": WORKLOAD_TEXT, "nx": sc.nx, "ny": sc.ny, "dx": sc.dx,
                       "n_peds": sc.n_peds, "n_responders": int((sc.peds["role"] == 1).sum()),
                       "barrier_cells": int(sc.barrier_cells.size), "barrier_layers": int(sc.n_layers),
                       "t0_s": sc.t0_ticks / float(1 << 20), "wet_fraction_at_start": float((sc.h > 0).mean()),
                       "sim_steps_per_bench_step": CHUNK,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed between timed iterations (256 MB write); the working set (~0.5 GB) "
                             "exceeds L2",
                       "tile_rows": tuned["tile_rows"], "ped_lanes": tuned["ped_lanes"],
                       "hash_ahead": tuned["hash_ahead"],
                       "launch_shape": "default" if args.no_tune else "fastest autotuner candidate on the snapshot"},
            "breakdown": {"cell_updates_per_s": steps_total * sc.n_cells / t_sec,
                          "computed_cell_updates_per_s": steps_total * flood_cells / t_sec,
                          "computed_cells_per_step": flood_cells, "cells_per_step": sc.n_cells,
                          "ped_updates_per_s": ped_total / t_sec,
                          "us_per_sim_step": 1e3 * ms_step / CHUNK,
                          "profiled_us_per_step": {k[:-3]: 1e3 * prof[k] / nprof
                                                   for k in ("hash_ms", "flood_ms", "ped_chain_ms", "ped_ms",
                                                             "step_ms")}},
            "roofline": {"kernel": "flood_kernel<%d>" % tuned["tile_rows"], "bound": "hbm", "achieved": achieved,
                         "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": flood_traffic(WORKLOAD), "bytes_per_cell_update": FLOOD_BYTES_PER_CELL,
                         "computed_cells_per_launch": flood_cells, "cells_per_launch": sc.n_cells,
                         "us_per_launch": flood_ms * 1e3,
                         "note": "launch duration from CUDA events on the flood kernel's own stream in a profiled "
                                 "pass of the same 512 steps; bytes counted for the cells of the tiles computed"},
            "roofline_peds": {"kernel": "ped_step_kernel<%d>" % tuned["ped_lanes"], "bound": "hbm",
                              "achieved": ped_achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                              "frac": ped_achieved / hbm if ped_achieved else None, "traffic": None,
                              "bytes_per_ped_update": PED_BYTES, "peds_per_launch": peds_per_step,
                              "us_per_launch": ped_ms * 1e3,
                              "note": "issue- and latency-bound (neighbour scans out of L1/L2); HBM fraction of "
                                      "its algorithmic bytes for reference"},
            "roofline_wet2048": roof_wet,
            "roofline_muscl_wet2048": roof_muscl,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "batched": batched,
            "surrogate": surrogate,
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
    """Learned surrogate against the plain update on the benchmark snapshot
    (2048x2048 shopping centre mid-flood, 100,000 coupled pedestrians), over
    --steps x 8 windows."""
    import torch
    import paper_1908_05232_b300 as P
    from paper_1908_05232_b300 import _native as N
    torch.cuda.set_device(0)
    P.build.build()
    args.surrogate_windows = args.steps * 8
    out = surrogate_figures(P, N, workload(3), args)
    line = {"metric": "scenario-seconds/s (learned surrogate windows vs plain update)", "value": out["value"],
            "unit": "scenario-s/s", "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 net (FP32 accumulate), f32 plain update",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (fixed 2^-5 s step)"}, "surrogate": out}
    print(json.dumps(line), flush=True)
    return 0


def run_ensemble(args):
    """Batched ensemble (--ensemble-size scenarios) against one by one."""
    import torch
    import paper_1908_05232_b300 as P
    torch.cuda.set_device(0)
    P.build.build()
    args.ensemble_steps = args.steps
    out = batched_figures(P, args, torch.device("cuda", 0))
    line = {"metric": "scenario-seconds/s (batched ensemble)", "value": out["value"], "unit": "scenario-s/s",
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ensemble_%d" % out["scenarios"]}, "batched": out}
    print(json.dumps(line), flush=True)
    return 0


def run_deployment(args):
    """Scenario 2 of the paper (Section 3.3): 6 responder group sizes x 6
    barrier thicknesses on the synthetic shopping centre at the paper's
    resolution (128 x 128 cells of 2.59 m, 1000 pedestrians), stepped as one
    batch until every barrier is built or 12 h have passed, then the
    (160 m^3/s, 7.5 min) discharge flood; prints the deployment table."""
    import torch
    import paper_1908_05232_b300 as P
    from paper_1908_05232_b300 import studies
    torch.cuda.set_device(0)
    P.build.build()
    t0 = time.perf_counter()
    res = studies.deployment_study(P, flood_minutes=args.deploy_flood_minutes)
    wall = time.perf_counter() - t0
    line = {"metric": "scenario-seconds/s (Section 3.3 deployment study as one batched ensemble)",
            "value": res["ensemble_sim_seconds"] / wall, "unit": "scenario-s/s", "n_gpus": 1, "steps": 1,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "deployment_36 (6 responder fractions x 6 layers, 128x128 "
                                                        "cells of 2.59 m, 1000 pedestrians, 12 h window)"},
            "wall_s": wall, "rows": res["rows"]}
    print(json.dumps(line), flush=True)
    return 0


def run_scenario1(args):
    """Scenario 1 of the paper (Section 3.2) on the synthetic shopping centre
    at the paper's resolution (128 x 128 cells of 2.59 m, 7 doors): visitors
    enter and leave through the doors during a 5-minute pre-flood spread, then
    the (160 m^3/s, 7.5 min) discharge flood enters, the first wet cell stops
    the entries and everyone present evacuates.  Runs with and without the
    evacuees' roughness coupling, each to the last evacuee out (or 1 h): whole
    run timed in 64-step chunks (the evacuee count polled after each), then the
    same run again sampling the flood-risk states every 0.1 min (Fig. 6).  The
    oracle is timed on the run's first steps, the GPU on the same steps."""
    import torch
    import scenarios
    import paper_1908_05232_b300 as P
    from paper_1908_05232_b300 import studies
    torch.cuda.set_device(0)
    P.build.build()
    T = 1 << 20
    pre, t_end = 300.0, 3600.0

    def make(coupling):
        return scenarios.scenario1(pre_flood=pre, period=args.s1_period, coupling=coupling, t_end=t_end)

    def run(sim, max_steps=None):
        steps = 0
        while True:
            k = 64 if max_steps is None else min(64, max_steps - steps)
            sim.step(k)
            steps += k
            c = sim.counters()  # synchronises
            if max_steps is not None and steps >= max_steps:
                return c
            if c["t_ticks"] >= int(t_end * T) or (c["t_ticks"] > int(pre * T) and c["wet"] and c["n_active"] == 0):
                return c

    warm = P.from_scenario(make(1))  # graphs and first-touch costs, not timed
    run(warm, 256)
    warm.close()
    runs = {}
    for coupling in (1, 0):
        sc = make(coupling)
        sim = P.from_scenario(sc)
        t0 = time.perf_counter()
        c = run(sim)
        wall = time.perf_counter() - t0
        sim.close()
        st = studies.evacuation_study(P, coupling, pre_flood=pre, period=args.s1_period, t_end=t_end)
        hist = np.array([h for _, _, h in st["samples"]])
        runs["with_coupling" if coupling else "without_coupling"] = {
            "wall_s": wall, "steps": int(c["step"]), "simulated_s": c["t_ticks"] / T,
            "scenario_s_per_s": c["t_ticks"] / T / wall, "steps_per_s": c["step"] / wall,
            "ped_updates_per_s": c["ped_updates"] / wall,
            "cell_updates_per_s": c["step"] * sc.nx * sc.ny / wall,
            "visitors_admitted": int(c["n_entered"]), "left_through_doors": int(c["n_left"]),
            "evacuated": int(c["n_exited"]), "population_at_flood": st["population_at_flood"],
            "evacuation_done_after_flood_s": st["evacuated_after_s"],
            "peak_per_state": {k: int(hist[:, i].max()) if hist.size else 0
                               for i, k in enumerate(("dry", "low", "medium", "high", "highest"))},
            "per_minute": [(round(t / 60.0, 2), n, h) for t, n, h in st["samples"][::10]]}
    # the oracle on the run's first steps (bounded), the GPU on the same steps
    import oracle
    oracle.build()
    o = oracle.Oracle(make(1))
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < args.s1_cpu_seconds:
        if o.step(8) < 8:
            break
        oc = o.flow_counts()
        if o.t_ticks > int(pre * T) and o.counters()["wet"] and oc["n_active"] == 0:
            break
    cpu_wall = time.perf_counter() - t0
    k = o.nstep
    sim = P.from_scenario(make(1))
    t0 = time.perf_counter()
    run(sim, k)
    gpu_wall = time.perf_counter() - t0
    sim.close()
    w = runs["with_coupling"]
    line = {"metric": "scenario-seconds/s (Section 3.2 Scenario 1: entry/exit flow, flood, evacuation)",
            "value": w["scenario_s_per_s"], "unit": "scenario-s/s", "n_gpus": 1, "steps": w["steps"],
            "warmup": 256, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "scenario1_128 (128x128 cells of 2.59 m, 7 doors, one visitor per door every "
                                   "%g s, 300 s pre-flood spread, (160 m^3/s, 7.5 min) discharge flood, to the last "
                                   "evacuee out or 1 h)" % args.s1_period},
            "runs": runs,
            "cpu_baseline": {"value": o.t_ticks / T / cpu_wall, "unit": "scenario-s/s", "cores": 1, "kind": "oracle",
                             "sample": "the run's first %d steps (t = 0 .. %.0f s)" % (k, o.t_ticks / T),
                             "gpu_same_steps_s": gpu_wall, "cpu_s": cpu_wall}}
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
    if args.ncu_case == "surrogate_forward":
        # the surrogate's tensor-core forward on 16 net input tiles of 266 x 266
        # pixels (a window's batch), twice; each forward launches the five
        # conv3x3_tc_kernel layers
        sur = P.Surrogate(seed=1)
        g = torch.Generator(device="cuda").manual_seed(1)
        x = torch.rand((16, 266, 266, 4), device="cuda", generator=g)
        y = torch.zeros((16, 256, 256, 3), device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sur.forward(x, y)
        e0.record()
        sur.forward(x, y)
        e1.record()
        torch.cuda.synchronize()
        flops = 16 * 266 * 266 * 73728
        print(json.dumps({"case": "surrogate_forward", "ms": e0.elapsed_time(e1),
                          "tflops_padded": flops / (e0.elapsed_time(e1) * 1e-3) / 1e12}))
        return 0
    if args.ncu_case == "surrogate_train":
        # Adam steps of the surrogate on a batch of 64 crops of 42 x 42 cells (the
        # training sampler's shape): forward, loss, the tensor-core backward
        # (weight and data gradients of the five layers), Adam, repacking;
        # --case-steps of them after two untimed
        sur = P.Surrogate(seed=1)
        g = torch.Generator(device="cuda").manual_seed(1)
        x = torch.rand((64, 42, 42, 4), device="cuda", generator=g)
        t = 0.05 * torch.randn((64, 32, 32, 3), device="cuda", generator=g)
        for _ in range(2):
            sur.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.case_steps):
            loss = sur.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        print(json.dumps({"case": "surrogate_train", "steps": args.case_steps, "loss": loss,
                          "ms_per_step": (time.perf_counter() - t0) * 1e3 / max(args.case_steps, 1)}))
        return 0
    if args.ncu_case == "barrier2048":
        sc = scenarios.config_barrier()
    elif args.ncu_case == "barrier2048mid":
        sc = workload(3)
    elif args.ncu_case == "wet2048":
        sc = wet2048()
    elif args.ncu_case == "wet1024":
        sc = scenarios.random_wet_state(1024, 1024, dx=0.5, seed=5)
    else:
        sc = scenarios.config_shopping()
    from paper_1908_05232_b300 import _native as N
    sc.order = args.case_order
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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--no-wet2048", action="store_true", help="skip the wet 2048x2048 flood-kernel roofline pass")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (16-row tiles, 8 lanes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-ensemble figures")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate figures")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--ref-budget-s", type=float, default=150.0,
                    help="reference arm: stop timing oracle steps once this many seconds are spent")
    ap.add_argument("--ensemble-size", type=int, default=48)
    ap.add_argument("--ensemble-steps", type=int, default=4, help="64-step chunks timed per ensemble arm")
    ap.add_argument("--surrogate-windows", type=int, default=160)
    ap.add_argument("--ncu-case", choices=["barrier2048", "barrier2048mid", "wet2048", "wet1024", "shopping512",
                                           "surrogate_forward", "surrogate_train"],
                    default=None, help="short untimed run of one workload, for profiler captures")
    ap.add_argument("--case-steps", type=int, default=4)
    ap.add_argument("--case-lanes", type=int, default=8, choices=[1, 2, 4, 8, 16], help="lanes per pedestrian in the case")
    ap.add_argument("--case-hash-ahead", type=int, default=1, choices=[0, 1], help="hash-ahead in the case")
    ap.add_argument("--case-order", type=int, default=1, choices=[1, 2],
                    help="flood update of the case: 1 first order, 2 the second-order option")
    ap.add_argument("--case-time", type=float, default=0.0,
                    help="simulated seconds to run before the case's steps (profiler range opened after them)")
    ap.add_argument("--workload", choices=["barrier2048", "ensemble", "surrogate", "deployment", "scenario1"],
                    default="barrier2048")
    ap.add_argument("--s1-period", type=float, default=1.25,
                    help="scenario1: seconds between admissions per door (1.25 s holds about 1000 visitors)")
    ap.add_argument("--s1-cpu-seconds", type=float, default=15.0, help="scenario1: oracle sample length (s)")
    ap.add_argument("--deploy-flood-minutes", type=float, default=20.0)
    args = ap.parse_args()
    if args.ncu_case:
        return run_case(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "deployment":
        return run_deployment(args)
    if args.workload == "scenario1":
        return run_scenario1(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
