"""Autotuner for the launch shape of a simulation and of a batched ensemble.

tune / choose: times every candidate (flood tile height 8/16/32, lanes per
pedestrian 1/2/4/8/16, hashing of the next step's records in the pedestrian
kernel or in a pass of its own, per-step kernels or the persistent kernel) for
a few dozen steps on a scratch copy of the scenario, picks the fastest and
caches the choice in a JSON file keyed by device, grid size and crowd size.

tune_batch: the shapes of a batch's members, raced on a scratch batch of the
same scenarios -- first one shape for all members, then, member size class by
size class, the shape of that class with the others held (coordinate
descent).  The candidates of a race are batches over the same members that
take turns, so all of them are timed on the same range of states.

The launch shape never changes the results (the same arithmetic runs in every
shape), only the time.
"""
from __future__ import annotations

import json
import os

from . import _native as N

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "floodped_autotune.json")
TILE_ROWS = (8, 16, 32)
PED_LANES = (1, 2, 4, 8, 16)
HASH_AHEAD = (True, False)


def cache_key(device: str, nx: int, ny: int, n_peds: int) -> str:
    bucket = 0 if n_peds == 0 else 1 << max(0, int(n_peds - 1).bit_length())
    return "%s|%dx%d|peds<=%d" % (device, nx, ny, bucket)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(sc, steps: int = 48, warm: int = 16, modes=(N.FP_MODE_KERNELS, N.FP_MODE_PERSISTENT)) -> dict:
    """Time every candidate on a scratch simulation of ``sc``; returns the
    fastest {"tile_rows", "ped_lanes", "hash_ahead", "mode", "us_per_step"} and
    all timings."""
    import torch
    stream = torch.cuda.Stream()
    sim = N.from_scenario(sc)
    N.fp_set_stream(sim.h, stream.cuda_stream)
    sim.step(warm)
    sim.synchronize()
    results = []
    for mode in modes:
        try:
            N.fp_set_step_mode(sim.h, mode)
        except N.FloodPedError:
            continue
        for rows in TILE_ROWS:
            for lanes in PED_LANES:
                for ahead in HASH_AHEAD:
                    if mode == N.FP_MODE_PERSISTENT and (rows != 8 or lanes != 1 or not ahead):
                        continue  # the persistent kernel has one fixed shape (8-row runs, 1 lane)
                    N.fp_set_tuning(sim.h, rows, lanes)
                    N.fp_set_hash_ahead(sim.h, ahead)
                    sim.step(8)
                    sim.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sim.step(steps)
                    e1.record(stream)
                    e1.synchronize()
                    results.append({"tile_rows": rows, "ped_lanes": lanes, "hash_ahead": ahead, "mode": mode,
                                    "us_per_step": 1e3 * e0.elapsed_time(e1) / steps})
    sim.close()
    best = min(results, key=lambda r: r["us_per_step"])
    return {"best": best, "all": results}


def choose(sc, cache_path: str = DEFAULT_CACHE, retune: bool = False) -> dict:
    """The cached best launch shape for ``sc`` on this device (tuning if absent)."""
    import torch
    key = cache_key(torch.cuda.get_device_name(), sc.nx, sc.ny, sc.n_peds)
    cache = _load(cache_path)
    if retune or key not in cache:
        cache[key] = tune(sc)["best"]
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = cache_path + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return cache[key]


def apply(sim, best: dict) -> None:
    N.fp_set_step_mode(sim.h, best["mode"])
    N.fp_set_tuning(sim.h, best["tile_rows"], best["ped_lanes"])
    N.fp_set_hash_ahead(sim.h, best.get("hash_ahead", True))


def size_classes(cells, classes: int = 2):
    """Class of each member (0 = smallest grids): members ranked by cell count
    (ties in input order), the member of rank r in class floor(r classes / n)
    -- groups of nearly equal size, the smaller grids taking any remainder."""
    n = len(cells)
    order = sorted(range(n), key=lambda k: cells[k])
    cls = [0] * n
    for rank, k in enumerate(order):
        cls[k] = min(classes - 1, rank * classes // max(n, 1))
    return cls


def _race(members, shape_lists, rounds: int = 2, chunk: int = 64):
    """Milliseconds per step of one batch per entry of ``shape_lists`` (per-member
    (tile_rows, ped_lanes)), all over the same ``members``: every batch is made
    and warmed (its step graph captured), then the batches take turns, ``rounds``
    chunks of ``chunk`` steps each, so that every candidate is timed on the
    same range of states of the advancing members."""
    import torch
    batches = []
    try:
        for shapes in shape_lists:
            for m, (rows, lanes) in zip(members, shapes):
                N.fp_set_tuning(m.h, rows, lanes)
            batches.append(N.Batch(members))
        for b in batches:
            b.step(chunk)
            b.synchronize()
        total = [0.0] * len(batches)
        for _ in range(rounds):
            for k, b in enumerate(batches):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                b.step(chunk)
                b.synchronize()
                e1.record()
                e1.synchronize()
                total[k] += e0.elapsed_time(e1)
        return [t / (rounds * chunk) for t in total]
    finally:
        for b in batches:
            b.close()


def tune_batch(scs, rounds: int = 3, classes: int = 2, margin: float = 0.02) -> dict:
    """Launch shapes for a batch of the scenarios ``scs`` (per-step-kernel mode),
    raced on a scratch batch: the 15 uniform shapes, then for each of
    ``classes`` member size classes (by cell count) the 15 shapes of that class
    with the others held, the incumbent among them (coordinate descent; a
    class moves only to a shape more than ``margin`` faster than its
    incumbent in the same race, so that race-to-race noise does not move it).
    Returns {"shapes": [(tile_rows, ped_lanes) per scenario], "us_per_step",
    "uniform": {shape: us}, "classes": [class of each scenario]}."""
    if not scs:
        return {"shapes": [], "us_per_step": 0.0, "uniform": {}, "classes": []}
    members = [N.from_scenario(sc) for sc in scs]
    try:
        n = len(scs)
        cls = size_classes([sc.nx * sc.ny for sc in scs], classes)
        cands = [(r, l) for r in TILE_ROWS for l in PED_LANES]
        ms = _race(members, [[c] * n for c in cands], rounds)
        uniform = {c: 1e3 * t for c, t in zip(cands, ms)}
        class_shape = [min(uniform, key=uniform.get)] * classes
        best = uniform[class_shape[0]]
        for c in range(classes):
            if c not in cls:
                continue  # no member of this size class
            trials = []
            for cand in cands:
                t = list(class_shape)
                t[c] = cand
                trials.append(t)
            ms = _race(members, [[t[cls[k]] for k in range(n)] for t in trials], rounds)
            k_inc = cands.index(class_shape[c])
            k_best = min(range(len(trials)), key=lambda k: ms[k])
            if ms[k_best] < (1.0 - margin) * ms[k_inc]:
                class_shape, best = trials[k_best], 1e3 * ms[k_best]
            else:
                best = 1e3 * ms[k_inc]
        return {"shapes": [class_shape[cls[k]] for k in range(n)], "us_per_step": best,
                "uniform": {"%dx%d" % k: v for k, v in uniform.items()}, "classes": cls}
    finally:
        for m in members:
            m.close()


def apply_batch(members, shapes) -> None:
    """Set each member's (tile_rows, ped_lanes) before the batch is made."""
    for m, (rows, lanes) in zip(members, shapes):
        N.fp_set_tuning(m.h, rows, lanes)
