"""FP64 CPU oracle of the coupled flood-pedestrian step -- TEST INFRASTRUCTURE.

This package wraps ``floodped_oracle.c`` (plain, single-threaded FP64 C, see its
header for the paper passages each function follows).  It is a checker, not a
product component: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library and never imports it.

Parity unpinned: the pedestrian repulsion constants (reading of the cited
social-force model) and the paper's 3484-bag barrier count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "floodped_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
TICKS = 1 << 20
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.or_step.restype = ctypes.c_int64
        _lib.or_run.restype = ctypes.c_int64
        _lib.or_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        _lib.or_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_prepare.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_mass.restype = ctypes.c_double
        _lib.or_mass.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_dt_ticks.restype = ctypes.c_int64
        _lib.or_dt_ticks.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64]
        _lib.or_hr_state.restype = ctypes.c_int
        _lib.or_hr_state.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float]
        _lib.or_hllc.restype = None
        _lib.or_hllc.argtypes = [ctypes.c_double] * 7 + [ctypes.c_void_p]
        _lib.or_hll.restype = None
        _lib.or_hll.argtypes = [ctypes.c_double] * 7 + [ctypes.c_void_p]
        _lib.or_philox4x64.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_visitor_draw.restype = None
        _lib.or_visitor_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_discharge.restype = ctypes.c_double
        _lib.or_discharge.argtypes = [ctypes.c_void_p, ctypes.c_double]
        _lib.or_discharge_volume.restype = ctypes.c_double
        _lib.or_discharge_volume.argtypes = [ctypes.c_void_p, ctypes.c_double]
        _lib.or_discharge_width.restype = ctypes.c_double
        _lib.or_discharge_width.argtypes = [ctypes.c_void_p]
        _lib.or_guard_residual.restype = ctypes.c_double
        _lib.or_guard_residual.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 7 + [ctypes.c_int32] * 4 + \
            [ctypes.c_int64] * 2
        _lib.or_max_hr.restype = ctypes.c_float
        _lib.or_max_hr.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_hydro_depth.restype = ctypes.c_double
        _lib.or_hydro_depth.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        _lib.or_nav_field.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_bags_per_cell.restype = ctypes.c_int32
        _lib.or_bags_per_cell.argtypes = [ctypes.c_double]
        _lib.or_flood_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        _lib.or_conv3x3.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        _lib.or_net_loss_grad.restype = ctypes.c_double
        _lib.or_net_loss_grad.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_int]
    return _lib


_P = ctypes.c_void_p


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dx", ctypes.c_double), ("g", ctypes.c_double), ("cfl", ctypes.c_double),
        ("t_end_ticks", ctypes.c_int64),
        ("n_hydro", ctypes.c_int32), ("hydro_t", _P), ("hydro_h", _P),
        ("bc_s", _P), ("bc_n", _P), ("bc_w", _P), ("bc_e", _P),
        ("n0", _P), ("walkable", _P), ("exit_mask", _P),
        ("n_depot", ctypes.c_int32), ("depot_cells", _P),
        ("n_barrier", ctypes.c_int32), ("barrier_cells", _P),
        ("n_layers", ctypes.c_int32), ("coupling", ctypes.c_int32), ("evac_trigger", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("ped_noise", ctypes.c_double), ("dt_fixed_ticks", ctypes.c_int64),
        ("n_q", ctypes.c_int32), ("q_t", _P), ("q_Q", _P), ("h_qin", ctypes.c_double),
        ("riemann", ctypes.c_int32),
        ("n_doors", ctypes.c_int32), ("n_door_cells", ctypes.c_int32), ("door_cells", _P), ("door_of", _P),
        ("entry_period_ticks", ctypes.c_int64), ("entry_v0_lo", ctypes.c_double), ("entry_v0_hi", ctypes.c_double),
        ("order", ctypes.c_int32),
    ]


class _State(ctypes.Structure):
    _fields_ = [
        ("h", _P), ("hu", _P), ("hv", _P), ("z", _P), ("bflux", _P),
        ("t_ticks", ctypes.c_int64), ("step", ctypes.c_int64),
        ("wet", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("total_bags", ctypes.c_int64), ("applied_layers", ctypes.c_int64),
        ("neg_depth", ctypes.c_int64), ("n_exited", ctypes.c_int64),
        ("hist", ctypes.c_int64 * 5),
        ("np", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("px", _P), ("py", _P), ("pvx", _P), ("pvy", _P), ("pv0", _P),
        ("pid", _P), ("ptimer", _P),
        ("prole", _P), ("pfsm", _P), ("phr", _P), ("pexit", _P),
        ("nav_exit", _P), ("nav_depot", _P), ("nav_barrier", _P),
        ("last_dt_ticks", ctypes.c_int64),
        ("cap", ctypes.c_int32), ("pad2", ctypes.c_int32),
        ("n_entered", ctypes.c_int64), ("n_left", ctypes.c_int64), ("entry_refused", ctypes.c_int64),
        ("nav_door", _P),
    ]


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _f32(v) -> float:
    """The FP32 value a scalar parameter takes on the GPU path, as a double."""
    return float(np.float32(v))


class Oracle:
    """Holds one scenario's state in FP64 and advances it with the C oracle."""

    def __init__(self, sc):
        L = lib()
        self.sc = sc
        nx, ny = sc.nx, sc.ny
        self._keep = []

        def keep(a):
            a = np.ascontiguousarray(a)
            self._keep.append(a)
            return a

        self.hydro_t = keep(np.asarray(sc.hydro_t, np.float64))
        self.hydro_h = keep(np.asarray(sc.hydro_h, np.float64))
        self.bc = [keep(np.asarray(b, np.uint8)) for b in (sc.bc_s, sc.bc_n, sc.bc_w, sc.bc_e)]
        self.n0 = keep(np.asarray(sc.n0, np.float64).reshape(-1))
        self.walkable = keep(np.asarray(sc.walkable, np.uint8).reshape(-1))
        self.exit_mask = keep(np.asarray(sc.exit_mask, np.uint8).reshape(-1))
        self.depot = keep(np.asarray(sc.depot_cells, np.int32))
        self.barrier = keep(np.asarray(sc.barrier_cells, np.int32))
        P = _Params()
        P.nx, P.ny = nx, ny
        P.dx, P.g, P.cfl = _f32(sc.dx), _f32(sc.g), _f32(sc.cfl)
        P.t_end_ticks = int(round(sc.t_end * TICKS))
        P.n_hydro = self.hydro_t.size
        P.hydro_t, P.hydro_h = _ptr(self.hydro_t), _ptr(self.hydro_h)
        P.bc_s, P.bc_n, P.bc_w, P.bc_e = [_ptr(b) for b in self.bc]
        P.n0, P.walkable, P.exit_mask = _ptr(self.n0), _ptr(self.walkable), _ptr(self.exit_mask)
        P.n_depot, P.depot_cells = self.depot.size, _ptr(self.depot)
        P.n_barrier, P.barrier_cells = self.barrier.size, _ptr(self.barrier)
        P.n_layers, P.coupling, P.evac_trigger = int(sc.n_layers), int(sc.coupling), int(sc.evac_trigger)
        P.seed = int(sc.seed) & ((1 << 64) - 1)
        P.ped_noise = _f32(sc.ped_noise)
        P.dt_fixed_ticks = int(getattr(sc, "dt_fixed_ticks", 0))
        self.q_t = keep(np.asarray(getattr(sc, "q_t", np.zeros(0)), np.float64))
        self.q_Q = keep(np.asarray(getattr(sc, "q_Q", np.zeros(0)), np.float64))
        P.n_q, P.q_t, P.q_Q = self.q_t.size, _ptr(self.q_t), _ptr(self.q_Q)
        P.h_qin = _f32(getattr(sc, "h_qin", 1.0))
        P.riemann = int(getattr(sc, "riemann", 0))
        self.door_cells = keep(np.asarray(getattr(sc, "door_cells", np.zeros(0)), np.int32))
        self.door_of = keep(np.asarray(getattr(sc, "door_of", np.zeros(0)), np.int32))
        P.n_doors = int(getattr(sc, "n_doors", 0))
        P.n_door_cells, P.door_cells, P.door_of = self.door_cells.size, _ptr(self.door_cells), _ptr(self.door_of)
        P.entry_period_ticks = int(round(float(getattr(sc, "entry_period", 6.0)) * TICKS))
        v0 = getattr(sc, "entry_v0", (1.4, 1.4))
        P.entry_v0_lo, P.entry_v0_hi = _f32(v0[0]), _f32(v0[1])
        P.order = int(getattr(sc, "order", 1))
        self.P = P
        n = nx * ny
        self.h = keep(np.asarray(sc.h, np.float64).reshape(-1).copy())
        self.hu = keep(np.asarray(sc.hu, np.float64).reshape(-1).copy())
        self.hv = keep(np.asarray(sc.hv, np.float64).reshape(-1).copy())
        self.z = keep(np.asarray(sc.z, np.float64).reshape(-1).copy())
        self.bflux = keep(np.zeros(2 * nx + 2 * ny, np.float64))
        p = sc.peds
        m = int(p["x"].shape[0])
        # room for the visitors the doors admit: ids up to the scenario's capacity
        cap = max(m, int(getattr(sc, "max_peds", 0) or 0))

        def grow(a, dtype):
            out = np.zeros(cap, dtype)
            out[:m] = a
            return keep(out)

        self.px = grow(p["x"], np.float64)
        self.py = grow(p["y"], np.float64)
        self.pvx = grow(p["vx"], np.float64)
        self.pvy = grow(p["vy"], np.float64)
        self.pv0 = grow(p["v0"], np.float64)
        self.pid = keep(np.arange(cap, dtype=np.int32))
        self.ptimer = grow(p["timer"], np.int32)
        self.prole = grow(p["role"], np.uint8)
        self.pfsm = grow(p["fsm"], np.uint8)
        self.phr = keep(np.zeros(cap, np.uint8))
        self.pexit = keep(np.zeros(cap, np.uint8))
        self.nav_exit = keep(np.zeros(n, np.uint8))
        self.nav_depot = keep(np.zeros(n, np.uint8))
        self.nav_barrier = keep(np.zeros(n, np.uint8))
        self.nav_door = keep(np.zeros(max(1, P.n_doors) * n, np.uint8))
        S = _State()
        S.h, S.hu, S.hv, S.z, S.bflux = [_ptr(a) for a in (self.h, self.hu, self.hv, self.z, self.bflux)]
        S.np = m
        S.px, S.py, S.pvx, S.pvy, S.pv0 = [_ptr(a) for a in (self.px, self.py, self.pvx, self.pvy, self.pv0)]
        S.pid, S.ptimer = _ptr(self.pid), _ptr(self.ptimer)
        S.prole, S.pfsm, S.phr, S.pexit = [_ptr(a) for a in (self.prole, self.pfsm, self.phr, self.pexit)]
        S.nav_exit, S.nav_depot, S.nav_barrier = _ptr(self.nav_exit), _ptr(self.nav_depot), _ptr(self.nav_barrier)
        S.nav_door, S.cap = _ptr(self.nav_door), cap
        S.t_ticks, S.step = int(sc.t0_ticks), int(sc.step0)
        S.total_bags, S.applied_layers = int(sc.bags0), int(sc.applied0)
        self.S = S
        L.or_prepare(ctypes.byref(P), ctypes.byref(S))

    # -- stepping ---------------------------------------------------------
    def step(self, n: int = 1) -> int:
        return int(lib().or_run(ctypes.byref(self.P), ctypes.byref(self.S), int(n)))

    def step_dt(self) -> int:
        return int(lib().or_step(ctypes.byref(self.P), ctypes.byref(self.S)))

    # -- views -----------------------------------------------------------
    @property
    def t(self) -> float:
        return self.S.t_ticks / TICKS

    @property
    def t_ticks(self) -> int:
        return int(self.S.t_ticks)

    @property
    def nstep(self) -> int:
        return int(self.S.step)

    def field(self, name):
        return getattr(self, name).reshape(self.sc.ny, self.sc.nx)

    def mass(self) -> float:
        return float(lib().or_mass(ctypes.byref(self.P), ctypes.byref(self.S)))

    def max_hr(self) -> float:
        """Largest hazard rating over the wet cells of the current state (FP32)."""
        return float(lib().or_max_hr(ctypes.byref(self.P), ctypes.byref(self.S)))

    def discharge(self, t: float) -> float:
        return float(lib().or_discharge(ctypes.byref(self.P), float(t)))

    def discharge_volume(self, t: float) -> float:
        return float(lib().or_discharge_volume(ctypes.byref(self.P), float(t)))

    def discharge_width(self) -> float:
        return float(lib().or_discharge_width(ctypes.byref(self.P)))

    def guard_residual(self, start, end, x0, x1, y0, y1, t0_ticks, t1_ticks) -> float:
        """The surrogate guard's mass residual of tile [x0, x1) x [y0, y1) for a
        window from state start = (h, hu, hv) at t0 to end at t1 (build-added
        check; the bed is this oracle's z)."""
        arrs = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in tuple(start) + tuple(end)]
        return float(lib().or_guard_residual(ctypes.byref(self.P), _ptr(self.z), *[_ptr(a) for a in arrs],
                                             int(x0), int(x1), int(y0), int(y1), int(t0_ticks), int(t1_ticks)))

    @property
    def n_peds(self) -> int:
        """Pedestrians ever in the domain (ids 0 .. n_peds - 1), present or gone."""
        return int(self.S.np)

    def flow_counts(self) -> dict:
        """Entry/exit flow counters: entered through the doors, left through
        their door, out through the emergency exit, refused for capacity, present."""
        S = self.S
        n = int(S.np)
        return dict(n_ids=n, n_entered=int(S.n_entered), n_left=int(S.n_left), n_exited=int(S.n_exited),
                    refused=int(S.entry_refused), n_active=n - int(S.n_left) - int(S.n_exited))

    def boundary_inflow(self) -> float:
        return float(self.bflux.sum())

    def dt_ticks_now(self) -> int:
        return int(lib().or_dt_ticks(ctypes.byref(self.P), _ptr(self.h), _ptr(self.hu), _ptr(self.hv),
                                     self.S.t_ticks))

    def counters(self) -> dict:
        S = self.S
        return dict(t_ticks=int(S.t_ticks), step=int(S.step), wet=int(S.wet), total_bags=int(S.total_bags),
                    applied_layers=int(S.applied_layers), neg_depth=int(S.neg_depth),
                    n_exited=int(S.n_exited), hist=[int(v) for v in S.hist],
                    n_active=int((self.pexit[:S.np] == 0).sum()))

    def to_scenario(self):
        """The oracle's current state as a new scenario (FP32-rounded fields and
        pedestrians still present, renumbered in id order), to start both
        implementations from one mid-run state."""
        import scenarios
        sc = self.sc.copy()
        ny, nx = sc.ny, sc.nx
        sc.h = self.h.reshape(ny, nx).astype(np.float32)
        sc.hu = self.hu.reshape(ny, nx).astype(np.float32)
        sc.hv = self.hv.reshape(ny, nx).astype(np.float32)
        sc.z = self.z.reshape(ny, nx).astype(np.float32)
        keep = np.zeros(self.pexit.size, bool)
        keep[:self.S.np] = self.pexit[:self.S.np] == 0
        p = scenarios.empty_peds(int(keep.sum()))
        p["x"], p["y"] = self.px[keep].astype(np.float32), self.py[keep].astype(np.float32)
        p["vx"], p["vy"] = self.pvx[keep].astype(np.float32), self.pvy[keep].astype(np.float32)
        p["role"], p["fsm"] = self.prole[keep].copy(), self.pfsm[keep].copy()
        p["timer"], p["v0"] = self.ptimer[keep].copy(), self.pv0[keep].astype(np.float32)
        sc.peds = p
        sc.t0_ticks, sc.step0 = int(self.S.t_ticks), int(self.S.step)
        sc.bags0, sc.applied0 = int(self.S.total_bags), int(self.S.applied_layers)
        return sc

    def peds(self) -> dict:
        """Every pedestrian so far by id (present or gone)."""
        n = int(self.S.np)
        return dict(x=self.px[:n].copy(), y=self.py[:n].copy(), vx=self.pvx[:n].copy(), vy=self.pvy[:n].copy(),
                    role=self.prole[:n].copy(), fsm=self.pfsm[:n].copy(), hr=self.phr[:n].copy(),
                    exited=self.pexit[:n].copy(), timer=self.ptimer[:n].copy(), v0=self.pv0[:n].copy())


# -- pointwise functions, used by the pins ------------------------------------
def hll(g, hL, unL, utL, hR, unR, utR):
    out = (ctypes.c_double * 3)()
    lib().or_hll(g, hL, unL, utL, hR, unR, utR, out)
    return np.array(out[:])


def hllc(g, hL, unL, utL, hR, unR, utR):
    out = (ctypes.c_double * 3)()
    lib().or_hllc(g, hL, unL, utL, hR, unR, utR, out)
    return np.array(out[:])


def hr_state(h, hu, hv) -> int:
    return int(lib().or_hr_state(h, hu, hv))


def philox4x64(counter, key):
    c = (ctypes.c_uint64 * 4)(*[int(v) & ((1 << 64) - 1) for v in counter])
    k = (ctypes.c_uint64 * 2)(*[int(v) & ((1 << 64) - 1) for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().or_philox4x64(c, k, o)
    return [int(v) for v in o]


def visitor_draw(seed, pid, n_doors, v0_lo, v0_hi):
    """A visitor's draws: (x offset, y offset) in cells inside its entry
    cell, dry walking speed (FP32 values) and destination door."""
    off = (ctypes.c_float * 3)()
    dest = ctypes.c_int32()
    lib().or_visitor_draw(int(seed) & ((1 << 64) - 1), int(pid), int(n_doors), float(np.float32(v0_lo)),
                          float(np.float32(v0_hi)), off, ctypes.byref(dest))
    return float(off[0]), float(off[1]), float(off[2]), int(dest.value)


def nav_field(walkable: np.ndarray, goal: np.ndarray):
    ny, nx = walkable.shape
    w = np.ascontiguousarray(walkable, np.uint8)
    gl = np.ascontiguousarray(goal, np.uint8)
    d = np.zeros((ny, nx), np.uint8)
    dist = np.zeros((ny, nx), np.int32)
    lib().or_nav_field(nx, ny, _ptr(w), _ptr(gl), _ptr(d), _ptr(dist))
    return d, dist


def bags_per_cell(dx: float) -> int:
    return int(lib().or_bags_per_cell(_f32(dx)))


# -- learned surrogate (build-added): FP64 conv net -----------------------------
def conv3x3(x, w, b, relu=False):
    """x: H x W x Ci, w: 3 x 3 x Ci x Co, b: Co -> (H-2) x (W-2) x Co (FP64)."""
    x = np.ascontiguousarray(x, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    H, W, Ci = x.shape
    Co = w.shape[3]
    y = np.zeros((H - 2, W - 2, Co), np.float64)
    lib().or_conv3x3(_ptr(x), H, W, Ci, _ptr(w), _ptr(b), Co, _ptr(y), 1 if relu else 0)
    return y


def net_forward(x, ws, bs):
    h = np.asarray(x, np.float64)
    for l, (w, b) in enumerate(zip(ws, bs)):
        h = conv3x3(h, w, b, relu=l + 1 < len(ws))
    return h


def net_loss_grad(x, ws, bs, target, act_bf16=False):
    """Mean squared error of the net output against target and its gradients.
    act_bf16: hidden activations stored rounded to BF16, as on the tensor-core
    path (the same ReLU decisions); False is the plain FP64 net."""
    x = np.ascontiguousarray(x, np.float64)
    H, W, _ = x.shape
    L = len(ws)
    ch = np.array([ws[0].shape[2]] + [w.shape[3] for w in ws], np.int32)
    ws_c = [np.ascontiguousarray(w, np.float64) for w in ws]
    bs_c = [np.ascontiguousarray(b, np.float64) for b in bs]
    n_act = sum((H - 2 * (l + 1)) * (W - 2 * (l + 1)) * int(ch[l + 1]) for l in range(L))
    acts = np.zeros(n_act, np.float64)
    big = max(H * W * int(c) for c in ch)
    scratch = np.zeros(2 * big, np.float64)
    dws = [np.zeros_like(w) for w in ws_c]
    dbs = [np.zeros_like(b) for b in bs_c]
    P = ctypes.c_void_p
    wp = (P * L)(*[w.ctypes.data for w in ws_c])
    bp = (P * L)(*[b.ctypes.data for b in bs_c])
    dwp = (P * L)(*[w.ctypes.data for w in dws])
    dbp = (P * L)(*[b.ctypes.data for b in dbs])
    tgt = np.ascontiguousarray(target, np.float64)
    loss = lib().or_net_loss_grad(_ptr(x), H, W, L, _ptr(ch), wp, bp, _ptr(tgt), _ptr(acts), dwp, dbp,
                                  _ptr(scratch), scratch.size, 1 if act_bf16 else 0)
    return float(loss), dws, dbs
