"""Seeded synthetic inputs for the coupled flood-pedestrian step.

This module only builds input arrays (terrain, boundary codes, hydrograph
tables, initial water state, pedestrian records) from a seed.  It holds none of
the method's arithmetic: no flux, no hazard rating, no pedestrian rule.  Both
the CUDA library binding and the FP64 oracle consume the ``Scenario`` objects it
returns, so it is the one piece of code the two share.

Workloads (all seeded, all synthetic):

* ``plain_coupled_128``  - 128x128 cells of 1 m, flat bed with a 1 m wall ring
  on the north/east/west sides and a 4-cell exit gap in the north wall, Manning
  n = 0.02, inflow along the south edge whose depth ramps 0 -> 0.5 m over 60 s,
  256 evacuees at uniform random dry positions (dry speed 1.2 m/s), 600 s.
* ``shopping_centre``  - a procedural stand-in for the paper's shopping centre
  (Section 3, Fig. 4, whose geometry is not available): a square domain with a
  wall ring, a central north-south corridor from the south breach to the north
  emergency exit, east-west cross corridors and 40-80 rectangular shop blocks
  (bed raised 2 m), +-2 cm bed noise, a triangular depth hydrograph on the
  south breach, evacuees seeded in the corridors, optionally responders, a
  sandbag depot and a barrier line across the corridor (Section 2.4).

Encodings shared with both implementations (an interface, not arithmetic):

* boundary codes per edge cell: 0 wall, 1 transmissive, 2 inflow (depth
  hydrograph), 3 discharge inflow (a wall through which the discharge
  hydrograph enters);
* pedestrian role: 0 evacuee, 1 responder; responder task state: 0 to depot,
  1 picking up, 2 to barrier, 3 dropping, 4 done; timers in ticks of 2**-20 s.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

BC_WALL, BC_TRANSMISSIVE, BC_INFLOW, BC_DISCHARGE = 0, 1, 2, 3
ROLE_EVACUEE, ROLE_RESPONDER = 0, 1
TICKS_PER_SECOND = 1 << 20


@dataclasses.dataclass
class Scenario:
    name: str
    nx: int
    ny: int
    dx: float
    t_end: float
    seed: int
    z: np.ndarray            # float32 [ny, nx], bed elevation (m)
    n0: np.ndarray           # float32 [ny, nx], base Manning n (s m^-1/3)
    walkable: np.ndarray     # uint8  [ny, nx]
    exit_mask: np.ndarray    # uint8  [ny, nx]
    bc_s: np.ndarray         # uint8  [nx]  south edge (row 0)
    bc_n: np.ndarray         # uint8  [nx]  north edge (row ny-1)
    bc_w: np.ndarray         # uint8  [ny]  west edge (column 0)
    bc_e: np.ndarray         # uint8  [ny]  east edge (column nx-1)
    hydro_t: np.ndarray      # float64 [k] times (s) of the depth hydrograph
    hydro_h: np.ndarray      # float64 [k] inflow depths (m)
    h: np.ndarray            # float32 [ny, nx] initial depth
    hu: np.ndarray           # float32 [ny, nx] initial x unit discharge
    hv: np.ndarray           # float32 [ny, nx] initial y unit discharge
    peds: dict               # x, y, vx, vy (f32), role, fsm (u8), timer (i32), v0 (f32)
    depot_cells: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    barrier_cells: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    n_layers: int = 0
    g: float = 9.81
    cfl: float = 0.5
    coupling: int = 1
    evac_trigger: int = 0
    ped_noise: float = 0.1
    t0_ticks: int = 0        # simulated time at the start (ticks of 2**-20 s)
    dt_fixed_ticks: int = 0  # > 0: every step this long (ticks), else the CFL step
    step0: int = 0           # step index at the start (random-generator counter)
    bags0: int = 0           # sandbags already dropped
    applied0: int = 0        # barrier cell-layers already built into z
    # discharge hydrograph through the boundary cells coded BC_DISCHARGE:
    # times (s), discharges Q (m^3/s), depth of the inflowing water (m)
    q_t: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    q_Q: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    h_qin: float = 1.0
    riemann: int = 0         # interface flux: 0 HLL, 1 HLLC
    order: int = 1           # 2: the second-order (MUSCL, two-stage) scheme
    # entrance doors (entry/exit flow before the flood): door_of[k] is the door
    # of cell door_cells[k] (a door's first listed cell is its entry cell); each
    # door admits one visitor every entry_period seconds, walking speeds drawn
    # in entry_v0 = (lo, hi) m/s; max_peds: pedestrian capacity (ids), 0 = the
    # initial count
    door_cells: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    door_of: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    n_doors: int = 0
    entry_period: float = 6.0
    entry_v0: tuple = (1.0, 1.6)
    max_peds: int = 0

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny

    @property
    def n_peds(self) -> int:
        return int(self.peds["x"].shape[0])

    def copy(self) -> "Scenario":
        out = dataclasses.replace(self)
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if isinstance(v, np.ndarray):
                setattr(out, f.name, v.copy())
        out.peds = {k: v.copy() for k, v in self.peds.items()}
        return out


def empty_peds(n: int = 0) -> dict:
    return dict(
        x=np.zeros(n, np.float32), y=np.zeros(n, np.float32),
        vx=np.zeros(n, np.float32), vy=np.zeros(n, np.float32),
        role=np.zeros(n, np.uint8), fsm=np.zeros(n, np.uint8),
        timer=np.zeros(n, np.int32), v0=np.zeros(n, np.float32))


def _place(rng: np.random.Generator, cells_ij: np.ndarray, n: int, dx: float) -> tuple:
    """n uniform positions inside cells drawn uniformly from ``cells_ij`` ([k, 2] = (i, j))."""
    if n == 0:
        return np.zeros(0, np.float32), np.zeros(0, np.float32)
    pick = rng.integers(0, cells_ij.shape[0], size=n)
    i = cells_ij[pick, 0].astype(np.float64)
    j = cells_ij[pick, 1].astype(np.float64)
    fx = rng.uniform(0.02, 0.98, size=n)
    fy = rng.uniform(0.02, 0.98, size=n)
    return ((i + fx) * dx).astype(np.float32), ((j + fy) * dx).astype(np.float32)


def _base(name, nx, ny, dx, t_end, seed) -> Scenario:
    return Scenario(
        name=name, nx=nx, ny=ny, dx=float(dx), t_end=float(t_end), seed=int(seed),
        z=np.zeros((ny, nx), np.float32), n0=np.full((ny, nx), 0.01, np.float32),
        walkable=np.ones((ny, nx), np.uint8), exit_mask=np.zeros((ny, nx), np.uint8),
        bc_s=np.zeros(nx, np.uint8), bc_n=np.zeros(nx, np.uint8),
        bc_w=np.zeros(ny, np.uint8), bc_e=np.zeros(ny, np.uint8),
        hydro_t=np.array([0.0]), hydro_h=np.array([0.0]),
        h=np.zeros((ny, nx), np.float32), hu=np.zeros((ny, nx), np.float32),
        hv=np.zeros((ny, nx), np.float32), peds=empty_peds(0))


# ---------------------------------------------------------------------------
# Benchmark-shaped workloads
# ---------------------------------------------------------------------------

def plain_coupled_128(seed: int = 1, n_peds: int = 256, nx: int = 128, ny: int = 128,
                      dx: float = 1.0, t_end: float = 600.0) -> Scenario:
    """Flat bed, 1 m wall ring (N/E/W), 4-cell exit gap, south inflow ramp 0->0.5 m in 60 s."""
    rng = np.random.default_rng(seed)
    s = _base("plain_coupled_128", nx, ny, dx, t_end, seed)
    s.n0[:] = 0.02
    s.z[ny - 1, :] = 1.0
    s.z[:, 0] = 1.0
    s.z[:, nx - 1] = 1.0
    gap0 = nx // 2 - 2
    s.z[ny - 1, gap0:gap0 + 4] = 0.0
    s.exit_mask[ny - 1, gap0:gap0 + 4] = 1
    s.walkable[:] = (s.z < 0.5).astype(np.uint8)
    s.bc_s[1:nx - 1] = BC_INFLOW
    s.bc_n[gap0:gap0 + 4] = BC_TRANSMISSIVE
    s.hydro_t = np.array([0.0, 60.0])
    s.hydro_h = np.array([0.0, 0.5])
    cand = np.argwhere((s.walkable == 1) & (s.exit_mask == 0))[:, ::-1]
    cand = cand[cand[:, 1] >= 1]                      # not on the inflow row
    p = empty_peds(n_peds)
    p["x"], p["y"] = _place(rng, cand, n_peds, dx)
    p["v0"][:] = 1.2
    s.peds = p
    s.evac_trigger = 0
    s.coupling = 1
    return s


def _shop_layout(rng, n, dx):
    """Wall ring, central corridor, cross corridors and 40-80 shop rectangles."""
    z = np.zeros((n, n), np.float32)
    shop = np.zeros((n, n), bool)
    L = n * dx
    z[n - 1, :] = 2.0
    z[:, 0] = 2.0
    z[:, n - 1] = 2.0
    z[0, :] = 2.0
    breach_w = int(round(min(100.0, 0.6 * L) / dx))
    b0 = n // 2 - breach_w // 2
    z[0, b0:b0 + breach_w] = 0.0
    exit_w = max(4, int(round(4.0 / dx)))
    e0 = n // 2 - exit_w // 2
    z[n - 1, e0:e0 + exit_w] = 0.0
    cw = int(round(0.3 * n))
    c0 = n // 2 - cw // 2
    c1 = c0 + cw
    cross_w = max(2, int(round(6.0 / dx)))
    gap = max(1, int(round(2.0 / dx)))
    n_rows = max(2, int(round(L / 40.0)))
    row_edges = np.linspace(2, n - 2, n_rows + 1).astype(int)
    target = int(rng.integers(40, 81))
    segments = []
    for r in range(n_rows):
        y0, y1 = row_edges[r] + cross_w // 2, row_edges[r + 1] - cross_w // 2
        if y1 - y0 < 2:
            continue
        segments.append((1 + gap, c0 - gap, y0, y1))
        segments.append((c1 + gap, n - 1 - gap, y0, y1))
    counts = np.full(len(segments), target // max(1, len(segments)), int)
    counts[: target - counts.sum()] += 1
    n_shops = 0
    for (x0, x1, y0, y1), k in zip(segments, counts):
        if k <= 0 or x1 - x0 < 2 * k:
            continue
        cuts = np.sort(rng.choice(np.arange(x0 + 1, x1), size=k - 1, replace=False)) if k > 1 else np.array([], int)
        edges = np.concatenate([[x0], cuts, [x1]])
        for a, b in zip(edges[:-1], edges[1:]):
            if b - a - gap < 1:
                continue
            shop[y0:y1, a:b - gap] = True
            n_shops += 1
    z[shop] += 2.0
    return z, shop, (b0, breach_w), (e0, exit_w), (c0, c1), n_shops


def shopping_centre(n: int = 512, dx: float = 0.5, n_evac: int = 10_000, n_resp: int = 0,
                    seed: int = 2, t_end: float = 1800.0, peak_depth: float = 1.0,
                    hydro=None, n_barrier: int = 0, n_layers: int = 0,
                    coupling: int = 1, evac_trigger: int = 1, discharge=None) -> Scenario:
    """Procedural shopping centre (stand-in for Fig. 4): see the module docstring."""
    rng = np.random.default_rng(seed)
    s = _base("shopping_centre_%d" % n, n, n, dx, t_end, seed)
    z, shop, (b0, bw), (e0, ew), (c0, c1), n_shops = _shop_layout(rng, n, dx)
    s.n_shops = n_shops
    s.breach = (b0, bw)
    ring = z >= 1.5
    noise = rng.uniform(-0.02, 0.02, size=(n, n)).astype(np.float32)
    s.z = (z + noise).astype(np.float32)
    s.walkable = (~ring).astype(np.uint8)
    s.exit_mask[n - 1, e0:e0 + ew] = 1
    s.bc_n[:] = BC_TRANSMISSIVE
    if discharge is None:
        s.bc_s[b0:b0 + bw] = BC_INFLOW
    else:
        # the paper's form (Section 3.1): a discharge hydrograph (q_peak, t_inflow)
        # through the breach, inflow depth 1 m; no depth hydrograph
        hydro = ([0.0], [0.0])
        with_discharge_breach(s, "south", b0, bw, discharge[0], discharge[1])
    if hydro is None:
        s.hydro_t = np.array([0.0, 300.0, 900.0])
        s.hydro_h = np.array([0.0, peak_depth, 0.0])
    else:
        s.hydro_t = np.asarray(hydro[0], np.float64)
        s.hydro_h = np.asarray(hydro[1], np.float64)
    s.n0[:] = 0.01
    s.coupling = coupling
    s.evac_trigger = evac_trigger
    corridor = np.argwhere((s.walkable == 1) & (s.exit_mask == 0))[:, ::-1]
    corridor = corridor[(corridor[:, 1] >= 2) & (corridor[:, 1] <= n - 3)]
    p = empty_peds(n_evac + n_resp)
    p["x"], p["y"] = _place(rng, corridor, n_evac + n_resp, dx)
    p["v0"][:] = 1.4
    p["role"][n_evac:] = ROLE_RESPONDER
    s.peds = p
    if n_barrier > 0:
        yb = int(0.6 * n)
        nb = min(n_barrier, c1 - c0)
        xb0 = (c0 + c1) // 2 - nb // 2
        s.barrier_cells = (yb * n + np.arange(xb0, xb0 + nb)).astype(np.int32)
        yd, xd = int(0.85 * n), (c0 + c1) // 2
        s.depot_cells = np.array([yd * n + xd, yd * n + xd + 1,
                                  (yd + 1) * n + xd, (yd + 1) * n + xd + 1], np.int32)
        s.n_layers = n_layers
    return s


def with_doors(s: Scenario, n_doors: int = 7, period: float = 6.0, v0=(1.0, 1.6),
               capacity: Optional[int] = None) -> Scenario:
    """Entrance doors of the shopping centre (Sections 3, 3.2: 7 doors at the
    ends of the corridors): one cell each, just inside the west or east wall
    (alternately) at the cross corridors between the shop rows, from the
    south; each admits one visitor every ``period`` seconds (10 per door per
    minute at the default) while no water has been seen.  ``capacity``: the
    pedestrian ids the run may use (default: the present crowd plus every
    door's admissions until t_end)."""
    n = s.nx
    L = n * s.dx
    n_rows = max(2, int(round(L / 40.0)))
    rows = list(np.linspace(2, n - 2, n_rows + 1).astype(int)[1:-1])
    cells = []
    for k in range(n_doors):
        west = k % 2 == 0
        row = rows[k % len(rows)] if rows else n // 2
        if k >= len(rows):
            west = not west
        col = 1 if west else n - 2
        # the nearest walkable cell of that wall's column, outward from the row
        for dy in range(0, s.ny):
            hit = [r for r in (row - dy, row + dy) if 0 <= r < s.ny and s.walkable[r, col]]
            if hit:
                row = hit[0]
                break
        c = row * n + col
        assert s.walkable[row, col] and c not in cells, "no walkable door cell"
        cells.append(c)
    s.door_cells = np.array(cells, np.int32)
    s.door_of = np.arange(n_doors, dtype=np.int32)
    s.n_doors = int(n_doors)
    s.entry_period = float(period)
    s.entry_v0 = (float(v0[0]), float(v0[1]))
    if capacity is None:
        capacity = s.n_peds + n_doors * (int(s.t_end / period) + 1)
    s.max_peds = int(capacity)
    s.evac_trigger = 1
    return s


def scenario1(n: int = 128, dx: float = 2.59, pre_flood: float = 300.0, q_peak: float = 160.0,
              t_inflow: float = 450.0, period: float = 1.25, coupling: int = 1, t_end: float = 3600.0,
              seed: int = 6, n_doors: int = 7) -> Scenario:
    """Scenario 1 (Section 3.2, during-flood evacuation) on the synthetic
    shopping centre at the paper's resolution: empty at t = 0, visitors enter
    through the doors during a pre-flood spread of ``pre_flood`` seconds (the
    paper's 5 minutes, Q = 0), then the (q_peak, t_inflow) triangular discharge
    flood enters through the south breach (depth 1 m); the first wet cell
    stops the entries and turns everyone present into an evacuee.  One visitor
    per door every 1.25 s holds about the paper's 1000 pedestrians in this
    layout by the flood's start (a visitor stays about 3 minutes; one every
    6 s, 10 per door per minute, holds about 220)."""
    sc = shopping_centre(n, dx, 0, 0, seed, t_end, discharge=(q_peak, t_inflow), coupling=coupling)
    sc.q_t, sc.q_Q = triangular_discharge(q_peak, t_inflow, t_start=pre_flood)
    sc.name = "scenario1_%d" % n
    return with_doors(sc, n_doors, period, capacity=n_doors * (int((pre_flood + t_inflow) / period) + 2))


def triangular_discharge(q_peak: float, t_inflow: float, t_start: float = 0.0):
    """A triangular discharge hydrograph (Section 3.1): 0 at t_start, q_peak
    (m^3/s) at t_start + t_inflow / 2, 0 from t_start + t_inflow on; returns the
    (times, discharges) points."""
    return (np.array([t_start, t_start + 0.5 * t_inflow, t_start + t_inflow], np.float64),
            np.array([0.0, q_peak, 0.0], np.float64))


def with_discharge_breach(s: Scenario, edge: str, first: int, width: int, q_peak: float, t_inflow: float,
                          h_inflow: float = 1.0, t_start: float = 0.0) -> Scenario:
    """Code ``width`` boundary cells of an edge ('south', 'north', 'west',
    'east') from index ``first`` as the discharge breach and give the scenario a
    triangular discharge hydrograph."""
    codes = {"south": s.bc_s, "north": s.bc_n, "west": s.bc_w, "east": s.bc_e}[edge]
    codes[first:first + width] = BC_DISCHARGE
    s.q_t, s.q_Q = triangular_discharge(q_peak, t_inflow, t_start)
    s.h_qin = float(h_inflow)
    return s


def breach_basin(n: int = 64, dx: float = 5.0, breach_cells: int = 20, q_peak: float = 160.0,
                 t_inflow: float = 450.0, t_end: float = 1e9, seed: int = 0) -> Scenario:
    """A flat, dry, walled square whose south edge has a discharge breach of
    ``breach_cells`` cells in its middle (100 m at the defaults), fed by a
    triangular hydrograph; the water has nowhere to leave."""
    s = _base("breach_basin", n, n, dx, t_end, seed)
    s.n0[:] = 0.01
    s.coupling = 0
    return with_discharge_breach(s, "south", n // 2 - breach_cells // 2, breach_cells, q_peak, t_inflow)


def config_plain(seed=1):
    """Plain coupled step, 128x128, 256 evacuees, 600 s."""
    return plain_coupled_128(seed)


def config_shopping(seed=2):
    """Synthetic shopping centre, 512x512 at 0.5 m, 10,000 evacuees, 1800 s."""
    return shopping_centre(512, 0.5, 10_000, 0, seed, 1800.0)


def config_barrier(seed=3):
    """Pre-flood barrier deployment: 2048x2048 at 0.5 m, 100,000 pedestrians of which
    500 responders, 200-cell barrier raised by 2 layers (0.5 m), flood at 900 s, 3600 s."""
    return shopping_centre(2048, 0.5, 99_500, 500, seed, 3600.0,
                           hydro=([0.0, 900.0, 1500.0, 2700.0], [0.0, 0.0, 1.0, 0.0]),
                           n_barrier=200, n_layers=2)


def config_barrier_midflood(seed=3, t0=1500.0, reach_m=300.0, depth_m=1.0, speed_m_s=0.6, bags=600):
    """The pre-flood barrier deployment workload (``config_barrier``) taken up
    mid-flood, as a synthetic state: at t0 (the inflow hydrograph's peak) the
    water surface falls linearly from ``depth_m`` above the breach centre to
    nothing ``reach_m`` away (so raised shop blocks stay dry), flowing radially
    away from the breach at up to ``speed_m_s``; the crowd stands where it was
    seeded; the responders are mid-deployment, each in a seeded task with a
    seeded wait, ``bags`` sandbags already dropped and the completed cell-layers
    already built into the bed.  Only input arrays are built here -- the flood
    and the crowd evolve from this state under the method itself."""
    s = config_barrier(seed)
    rng = np.random.default_rng(seed + 104729)
    n = s.nx
    b0, bw = s.breach
    xc = (b0 + 0.5 * bw) * s.dx
    yy, xx = np.mgrid[0:n, 0:n]
    x = (xx + 0.5) * s.dx
    y = (yy + 0.5) * s.dx
    d = np.hypot(x - xc, y)
    eta = depth_m * np.clip(1.0 - d / reach_m, 0.0, None)
    h = np.maximum(eta - s.z.astype(np.float64), 0.0)
    h[s.z >= 1.0] = 0.0          # walls and shop blocks
    h[d >= reach_m] = 0.0        # beyond the front the floor is dry (no water in the bed noise's hollows)
    sp = speed_m_s * np.clip(1.0 - d / reach_m, 0.0, None)
    ux = np.where(d > 0, (x - xc) / np.maximum(d, 1e-9), 0.0) * sp
    uy = np.where(d > 0, y / np.maximum(d, 1e-9), 0.0) * sp
    s.h = h.astype(np.float32)
    s.hu = (s.h * ux).astype(np.float32)
    s.hv = (s.h * uy).astype(np.float32)
    s.h[s.h < 1e-4] = 0.0
    s.hu[s.h == 0] = 0.0
    s.hv[s.h == 0] = 0.0
    # responders mid-deployment
    resp = np.nonzero(s.peds["role"] == ROLE_RESPONDER)[0]
    s.peds["fsm"][resp] = rng.integers(0, 4, resp.size).astype(np.uint8)
    waiting = (s.peds["fsm"][resp] == 1) | (s.peds["fsm"][resp] == 3)
    s.peds["timer"][resp] = np.where(waiting, rng.integers(1, 30 * TICKS_PER_SECOND, resp.size), 0).astype(np.int32)
    bpc = int(np.ceil(float(np.float32(s.dx)) ** 2 / (0.40 * 0.30)))
    s.bags0 = int(bags)
    s.applied0 = min(int(bags) // bpc, s.barrier_cells.size * s.n_layers)
    for k in range(s.applied0):
        c = s.barrier_cells[k % s.barrier_cells.size]
        s.z.flat[c] += np.float32(0.25)
    s.t0_ticks = int(round(t0 * TICKS_PER_SECOND))
    s.step0 = 12_000
    s.name = "barrier_2048_midflood"
    return s


# ---------------------------------------------------------------------------
# Small cases for pins and parity tests
# ---------------------------------------------------------------------------

def closed_basin(nx, ny, dx=1.0, seed=0, wet=True, bumps=True, t_end=1e9) -> Scenario:
    """All-wall box with a seeded bed and water; used for mass and lake-at-rest tests.

    Bed values and the water level are multiples of 2**-12 m so that h + z is
    exactly the level in FP32 for every wet cell."""
    rng = np.random.default_rng(seed)
    s = _base("closed_basin", nx, ny, dx, t_end, seed)
    q = 2.0 ** -12
    if bumps:
        zz = rng.uniform(0.0, 0.6, size=(ny, nx))
        yy, xx = np.mgrid[0:ny, 0:nx]
        zz += 0.9 * np.exp(-(((xx - nx * 0.3) / (0.1 * nx + 1)) ** 2 + ((yy - ny * 0.6) / (0.1 * ny + 1)) ** 2))
        s.z = (np.round(zz / q) * q).astype(np.float32)
    eta = np.float32(0.75)
    if wet:
        s.h = np.maximum(eta - s.z, 0).astype(np.float32)
    s.n0[:] = 0.02
    s.peds = empty_peds(0)
    s.coupling = 0
    return s


def dam_break_1d(nx=400, ny=4, dx=0.25, h_left=1.0, h_right=0.0, x0_frac=0.5, t_end=10.0) -> Scenario:
    """Frictionless flat-bed dam break along x (Ritter if h_right = 0, Stoker otherwise)."""
    s = _base("dam_break", nx, ny, dx, t_end, 0)
    i0 = int(nx * x0_frac)
    s.h[:, :i0] = h_left
    s.h[:, i0:] = h_right
    s.n0[:] = 0.0
    s.bc_w[:] = BC_TRANSMISSIVE
    s.bc_e[:] = BC_TRANSMISSIVE
    s.coupling = 0
    return s


def random_wet_state(nx, ny, dx=1.0, seed=0, dry_frac=0.3, vel=1.5, t_end=1e9,
                     bc=(BC_WALL, BC_TRANSMISSIVE, BC_WALL, BC_INFLOW)) -> Scenario:
    """Seeded rough water state with dry patches, uneven bed and all boundary types.

    ``bc`` gives the codes of the south, north, west and east edges."""
    rng = np.random.default_rng(seed)
    s = _base("random_wet", nx, ny, dx, t_end, seed)
    s.z = rng.uniform(0.0, 0.5, size=(ny, nx)).astype(np.float32)
    h = rng.uniform(0.0, 1.2, size=(ny, nx))
    h[rng.uniform(size=(ny, nx)) < dry_frac] = 0.0
    s.h = h.astype(np.float32)
    s.hu = (s.h * rng.uniform(-vel, vel, size=(ny, nx))).astype(np.float32)
    s.hv = (s.h * rng.uniform(-vel, vel, size=(ny, nx))).astype(np.float32)
    s.n0 = rng.uniform(0.005, 0.05, size=(ny, nx)).astype(np.float32)
    s.bc_s[:], s.bc_n[:], s.bc_w[:], s.bc_e[:] = bc
    s.hydro_t = np.array([0.0, 5.0, 20.0])
    s.hydro_h = np.array([0.3, 0.9, 0.2])
    s.coupling = 0
    return s


def random_crowd(s: Scenario, n_evac: int, n_resp: int = 0, seed: int = 0,
                 v0=1.4, random_velocity=0.0, random_tasks=False) -> Scenario:
    """Add seeded pedestrians at uniform positions over walkable, non-exit cells."""
    rng = np.random.default_rng(seed + 7919)
    cand = np.argwhere((s.walkable == 1) & (s.exit_mask == 0))[:, ::-1]
    n = n_evac + n_resp
    p = empty_peds(n)
    p["x"], p["y"] = _place(rng, cand, n, s.dx)
    p["v0"][:] = v0
    p["role"][n_evac:] = ROLE_RESPONDER
    if random_velocity > 0:
        p["vx"] = rng.uniform(-random_velocity, random_velocity, n).astype(np.float32)
        p["vy"] = rng.uniform(-random_velocity, random_velocity, n).astype(np.float32)
    if random_tasks and n_resp:
        p["fsm"][n_evac:] = rng.integers(0, 5, n_resp).astype(np.uint8)
        p["timer"][n_evac:] = rng.integers(1, 40 * TICKS_PER_SECOND, n_resp).astype(np.int32)
    s.peds = p
    return s


def with_depot_and_barrier(s: Scenario, depot_ij, barrier_ij, n_layers) -> Scenario:
    s.depot_cells = np.array([j * s.nx + i for i, j in depot_ij], np.int32)
    s.barrier_cells = np.array([j * s.nx + i for i, j in barrier_ij], np.int32)
    s.n_layers = int(n_layers)
    return s


def ensemble(n: int = 256, seed: int = 4, side_range=(128, 1024), peds_range=(1_000, 50_000),
             resp_range=(50, 1_000), barrier_m=(0.2, 0.8), peak_m=(0.3, 1.5), dx: float = 0.5,
             t_end: float = 3600.0) -> list:
    """Seeded ensemble of shopping-centre scenarios: grid side log-uniform in
    side_range (multiple of 8), pedestrians uniform in peds_range of which
    responders uniform in resp_range, barrier height uniform in barrier_m
    (rounded to whole 0.25 m sandbag layers, at least one), inflow peak depth
    uniform in peak_m."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        side = int(np.exp(rng.uniform(np.log(side_range[0]), np.log(side_range[1]))))
        side = max(64, (side // 8) * 8)
        n_peds = int(rng.integers(peds_range[0], peds_range[1] + 1))
        n_resp = min(int(rng.integers(resp_range[0], resp_range[1] + 1)), n_peds // 2)
        layers = max(1, int(round(rng.uniform(*barrier_m) / 0.25)))
        peak = float(rng.uniform(*peak_m))
        # keep the crowd below ~1 pedestrian per square metre of the domain
        n_peds = min(n_peds, int((side * dx) ** 2 * 0.5))
        n_resp = min(n_resp, n_peds // 2)
        sc = shopping_centre(side, dx, n_peds - n_resp, n_resp, seed * 1000 + k, t_end,
                             hydro=([0.0, 300.0, 900.0], [0.0, peak, 0.0]),
                             n_barrier=min(200, side // 4), n_layers=layers)
        sc.name = "ensemble_%d" % k
        out.append(sc)
    return out
