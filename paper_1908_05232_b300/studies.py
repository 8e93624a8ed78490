"""Studies of the paper run on the batched ensemble (Section 3.3) and the
discharge hydrographs (Section 3.1), driving the C ABI; every simulation step
runs in the library's kernels, this module only sets up scenarios, steps the
batch and reads results back.

deployment_study -- Scenario 2 (pre-flood intervention, Section 3.3): responder
    groups of 5-50 % of the pedestrians build a sandbag barrier of 1-6 layers;
    all 6 x 6 runs stepped together as one batch until every barrier is built
    or the 12 h window has passed (Fig. 8: deployment time against the window),
    then each run takes the (160 m^3/s, 7.5 min) discharge flood through the
    breach, and the water depth along the corridor centreline downstream of the
    barrier and the largest hazard rating there are recorded (Figs. 9-10).
hr_history -- the maximum hazard rating over the domain sampled every 0.1 min
    under a discharge hydrograph (Fig. 5(b)).
evacuation_study -- Scenario 1 (during-flood evacuation, Section 3.2): visitors
    enter and leave through the doors during a pre-flood spread, the discharge
    flood enters, the first wet cell stops the entries and everyone present
    evacuates through the emergency exit; the pedestrians in each flood-risk
    state are counted every 0.1 min until the last one is out (Fig. 6), with
    and without the evacuees' effect on the local roughness.
"""
from __future__ import annotations

import numpy as np

from . import _native as N

PAPER_FRACTIONS = (0.05, 0.10, 0.20, 0.30, 0.40, 0.50)  # Section 3.3 responder group sizes
PAPER_LAYERS = (1, 2, 3, 4, 5, 6)                       # Section 3.3 barrier thicknesses
FLOOD = (160.0, 450.0)                                  # Section 3.1: (Q_peak m^3/s, t_inflow s) of Scenarios 1-2


def deployment_scenarios(fractions=PAPER_FRACTIONS, layers=PAPER_LAYERS, n=128, dx=2.59, n_peds=1000,
                         n_barrier=65, seed=5, window_h=12.0):
    """One scenario per (responder fraction, layers): the synthetic shopping
    centre at the paper's resolution (128 x 128 cells of 2.59 m, 1000
    pedestrians), the barrier across the corridor (as long as the corridor is
    wide, at most n_barrier cells), dry until the flood."""
    import scenarios
    out = []
    for f in fractions:
        n_resp = int(round(f * n_peds))
        for nl in layers:
            sc = scenarios.shopping_centre(n, dx, n_peds - n_resp, n_resp, seed, 3 * 3600.0 * window_h,
                                           hydro=([0.0], [0.0]), n_barrier=n_barrier, n_layers=nl)
            sc.name = "deploy_%02d%%_%dL" % (round(100 * f), nl)
            out.append((sc, dict(fraction=f, responders=n_resp, layers=nl)))
    return out


def _downstream(sc):
    """Rows north of the barrier (toward the exit) and the corridor columns the
    barrier spans: the region the flood reaches past it."""
    cells = np.asarray(sc.barrier_cells)
    yb = int(cells[0] // sc.nx)
    xs = cells % sc.nx
    return yb, int(xs.min()), int(xs.max()) + 1


def deployment_study(P, fractions=PAPER_FRACTIONS, layers=PAPER_LAYERS, n=128, dx=2.59, n_peds=1000, n_barrier=65,
                     seed=5, window_h=12.0, flood_minutes=20.0, poll_steps=64, sample_steps=32):
    """Runs the study; returns one row per run: fraction, responders, layers,
    deployment time (s; None if the window passed first), within the window,
    the largest depth on the corridor centreline downstream of the barrier and
    the largest hazard rating downstream during the flood, and the simulated
    seconds of the whole ensemble (for throughput)."""
    runs = deployment_scenarios(fractions, layers, n, dx, n_peds, n_barrier, seed, window_h)
    sims = [P.from_scenario(sc) for sc, _ in runs]
    batch = P.Batch(sims)
    window = window_h * 3600.0
    done = [None] * len(sims)
    target = [len(sc.barrier_cells) * sc.n_layers for sc, _ in runs]
    t_now = 0.0
    while True:
        batch.step(poll_steps)
        batch.synchronize()
        cs = [s.counters() for s in sims]
        t_now = min(c["t_ticks"] for c in cs) / N.TICKS
        for k, c in enumerate(cs):
            if done[k] is None and c["applied_layers"] >= target[k]:
                done[k] = c["t_ticks"] / N.TICKS
        if all(d is not None for d in done) or t_now >= window:
            break
    # the flood through the breach, from each run's present time on
    q_peak, t_inflow = FLOOD
    for (sc, _), sim in zip(runs, sims):
        t0 = sim.counters()["t_ticks"] / N.TICKS
        codes = np.asarray(sc.bc_s, np.uint8).copy()
        b0, bw = sc.breach
        codes[b0:b0 + bw] = N.FP_BC_DISCHARGE
        N.fp_set_boundary(sim.h, N.FP_EDGE_SOUTH, codes)
        N.fp_set_discharge(sim.h, [t0, t0 + 0.5 * t_inflow, t0 + t_inflow], [0.0, q_peak, 0.0], 1.0)
    t_start = [s.counters()["t_ticks"] for s in sims]
    regions = [_downstream(sc) for sc, _ in runs]
    depth = np.zeros(len(sims))
    hrmax = np.zeros(len(sims))
    flood_ticks = int(flood_minutes * 60.0 * N.TICKS)
    while True:
        batch.step(sample_steps)
        batch.synchronize()
        fin = True
        for k, sim in enumerate(sims):
            c = sim.counters()
            if c["t_ticks"] - t_start[k] < flood_ticks:
                fin = False
            yb, xa, xb = regions[k]
            h = sim.field(N.FP_FIELD_H)
            hu = sim.field(N.FP_FIELD_HU)
            hv = sim.field(N.FP_FIELD_HV)
            xc = (xa + xb) // 2
            depth[k] = max(depth[k], float(h[yb + 1:, xc].max()))
            hd = h[yb + 1:, xa:xb].astype(np.float32)
            wet = hd > np.float32(1e-6)
            if wet.any():
                V = np.maximum(np.abs(hu[yb + 1:, xa:xb][wet]), np.abs(hv[yb + 1:, xa:xb][wet])) / hd[wet]
                hrmax[k] = max(hrmax[k], float(((V + np.float32(0.5)) * hd[wet]).max()))
        if fin:
            break
    sim_seconds = sum(s.counters()["t_ticks"] for s in sims) / N.TICKS
    batch.close()
    rows = []
    for k, (sc, meta) in enumerate(runs):
        rows.append(dict(meta, deploy_s=done[k], within_window=done[k] is not None and done[k] <= window,
                         barrier_cells=int(len(sc.barrier_cells)), bags=int(target[k] * N_bags_per_cell(sc.dx)),
                         downstream_depth_m=float(depth[k]), downstream_max_hr=float(hrmax[k])))
    for s in sims:
        s.close()
    return dict(rows=rows, ensemble_sim_seconds=sim_seconds)


def N_bags_per_cell(dx):
    """Sandbags (40 x 30 cm, Section 3) covering one cell of side dx once."""
    return int(np.ceil(float(np.float32(dx)) ** 2 / (0.40 * 0.30)))


def hr_history(P, sc, minutes=60.0, every_s=6.0):
    """The largest hazard rating over the domain every every_s seconds (the
    paper records every 0.1 min) for minutes of simulated time (Fig. 5(b))."""
    sim = P.from_scenario(sc)
    out = []
    t_end = int(minutes * 60.0 * N.TICKS)
    nxt = int(every_s * N.TICKS)
    while True:
        c = sim.counters()
        if c["t_ticks"] >= t_end:
            break
        while sim.counters()["t_ticks"] < nxt:
            sim.step(1)
        out.append((sim.counters()["t_ticks"] / N.TICKS, sim.max_hr()))
        nxt += int(every_s * N.TICKS)
    sim.close()
    return out


def evacuation_study(P, coupling=1, n=128, dx=2.59, pre_flood=300.0, period=6.0, t_end=3600.0, seed=6,
                     every_s=6.0):
    """Scenario 1 on the synthetic shopping centre at the paper's resolution:
    returns the population when the flood started, the evacuation's end time
    after it (None if evacuees remain at t_end), the samples (t - pre_flood,
    pedestrians present, counts per flood-risk state of the last step) every
    every_s seconds from the flood's start, and the steps taken."""
    import scenarios
    sc = scenarios.scenario1(n, dx, pre_flood, period=period, coupling=coupling, t_end=t_end, seed=seed)
    sim = P.from_scenario(sc)
    t0 = int(pre_flood * N.TICKS)
    nxt = t0
    samples, pop0, done = [], None, None
    while True:
        c = sim.counters()
        t = c["t_ticks"]
        if t >= int(t_end * N.TICKS):
            break
        if t >= t0 and pop0 is None:
            pop0 = c["n_active"]
        if t >= nxt:
            samples.append(((t - t0) / N.TICKS, c["n_active"], list(c["hist"])))
            nxt += int(every_s * N.TICKS)
            if t > t0 and c["wet"] and c["n_active"] == 0:
                done = (t - t0) / N.TICKS
                break
        # steps are at most 1 s long: chunks that cannot pass the next sample
        sim.step(max(1, min(64, (nxt - t) // N.TICKS - 1)))
    steps = sim.counters()["step"]
    sim.close()
    return dict(population_at_flood=pop0, evacuated_after_s=done, samples=samples, steps=int(steps),
                coupling=int(coupling))
