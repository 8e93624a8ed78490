"""ctypes binding of ``libfloodped.so`` (include/floodped.h).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of the library.  Arrays may be numpy arrays (host) or CUDA torch
tensors (device); the library copies them.  If the library is missing the
import of a simulation fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FP_OK, FP_EINVAL, FP_ENOMEM, FP_ECUDA, FP_ETIMEOUT, FP_ENAN, FP_EOVERFLOW = 0, -1, -2, -3, -4, -5, -6
FP_FIELD_H, FP_FIELD_HU, FP_FIELD_HV, FP_FIELD_Z = 0, 1, 2, 3
FP_FIELD_PEDS, FP_FIELD_COUNTERS, FP_FIELD_NAV, FP_FIELD_MASS, FP_FIELD_PROFILE = 4, 5, 6, 7, 8
FP_FIELD_HR_MAX = 9
FP_BC_WALL, FP_BC_TRANSMISSIVE, FP_BC_INFLOW, FP_BC_DISCHARGE = 0, 1, 2, 3
FP_EDGE_SOUTH, FP_EDGE_NORTH, FP_EDGE_WEST, FP_EDGE_EAST = 0, 1, 2, 3
TICKS = 1 << 20
FP_MODE_KERNELS, FP_MODE_PERSISTENT = 0, 1

PED_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("vx", "<f4"), ("vy", "<f4"), ("id", "<u4"),
                      ("role", "u1"), ("task", "u1"), ("hr", "u1"), ("exited", "u1"),
                      ("timer_ticks", "<i4"), ("v0", "<f4")])
assert PED_DTYPE.itemsize == 32


class FpConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_float), ("g", ctypes.c_float),
                ("cfl", ctypes.c_float), ("ped_noise", ctypes.c_float), ("t_end", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("max_peds", ctypes.c_int32), ("coupling", ctypes.c_int32),
                ("evac_trigger", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("riemann", ctypes.c_int32),
                ("order", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class FpCounters(ctypes.Structure):
    _fields_ = [("t_ticks", ctypes.c_int64), ("step", ctypes.c_int64), ("n_active", ctypes.c_int64),
                ("n_exited", ctypes.c_int64), ("total_bags", ctypes.c_int64), ("applied_layers", ctypes.c_int64),
                ("neg_depth", ctypes.c_int64), ("hist", ctypes.c_int64 * 5), ("wet", ctypes.c_int32),
                ("error_flags", ctypes.c_uint32), ("ped_updates", ctypes.c_int64), ("cfl_exceeded", ctypes.c_int64),
                ("n_ids", ctypes.c_int64), ("n_entered", ctypes.c_int64), ("n_left", ctypes.c_int64)]


class SurGuard(ctypes.Structure):
    _fields_ = [("mass_tol", ctypes.c_float), ("check_tol", ctypes.c_float), ("check_every", ctypes.c_int32),
                ("suspend_windows", ctypes.c_int32), ("fix_tol", ctypes.c_float)]


class SurStats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_int64), ("tiles", ctypes.c_int64), ("tiles_net", ctypes.c_int64),
                ("tiles_fallback", ctypes.c_int64), ("fail_mass", ctypes.c_int64), ("fail_courant", ctypes.c_int64),
                ("fail_nonfinite", ctypes.c_int64), ("tiles_plain", ctypes.c_int64), ("checks", ctypes.c_int64),
                ("checks_failed", ctypes.c_int64), ("max_residual", ctypes.c_double),
                ("max_check_error", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FloodPedError(RuntimeError):
    pass


_lib = None
_VP = ctypes.c_void_p


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise FloodPedError("libfloodped.so is not built: run paper_1908_05232_b300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        sigs = {
            "fp_sim_create": [_VP, _VP], "fp_set_stream": [_VP, _VP],
            "fp_set_terrain": [_VP] * 5, "fp_set_bed": [_VP, _VP], "fp_set_boundary": [_VP, ctypes.c_int32, _VP],
            "fp_set_hydrograph": [_VP, _VP, _VP, ctypes.c_int32],
            "fp_set_discharge": [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_double],
            "fp_set_goals": [_VP, _VP, ctypes.c_int32, _VP, ctypes.c_int32, ctypes.c_int32],
            "fp_set_doors": [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double],
            "fp_set_state": [_VP] * 4, "fp_set_time": [_VP, ctypes.c_int64, ctypes.c_int64],
            "fp_set_barrier_progress": [_VP, ctypes.c_int64, ctypes.c_int64],
            "fp_add_pedestrians": [_VP, _VP, ctypes.c_int32], "fp_clear_pedestrians": [_VP],
            "fp_step": [_VP, ctypes.c_int32], "fp_synchronize": [_VP], "fp_set_step_mode": [_VP, ctypes.c_int32],
            "fp_set_tuning": [_VP, ctypes.c_int32, ctypes.c_int32], "fp_set_hash_ahead": [_VP, ctypes.c_int32],
            "fp_batch_create": [_VP, ctypes.c_int32, _VP], "fp_batch_step": [_VP, ctypes.c_int32],
            "fp_batch_synchronize": [_VP], "fp_batch_destroy": [_VP], "fp_set_profiling": [_VP, ctypes.c_int32],
            "fp_batch_set_step_mode": [_VP, ctypes.c_int32],
            "fp_read_state": [_VP, ctypes.c_int32, _VP, ctypes.c_size_t], "fp_destroy": [_VP],
            "fp_set_fixed_dt": [_VP, ctypes.c_double], "fp_set_barrier_wait_limit": [_VP, ctypes.c_int32], "fp_surrogate_advance": [_VP, _VP, ctypes.c_int32, _VP, _VP],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fp_water_volume_noalloc.argtypes = [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                              _VP, _VP]
        L.fp_water_volume_noalloc.restype = ctypes.c_int
        for name, args in {"fp_surrogate_create": [ctypes.c_uint64, _VP], "fp_surrogate_destroy": [_VP],
                           "fp_surrogate_get_params": [_VP, _VP, ctypes.c_size_t],
                           "fp_surrogate_set_params": [_VP, _VP, ctypes.c_size_t],
                           "fp_surrogate_forward": [_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP],
                           "fp_surrogate_num_params": [],
                           "fp_surrogate_gradients": [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                      _VP, _VP],
                           "fp_surrogate_train_step": [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                       ctypes.c_float, _VP],
                           "fp_surrogate_set_max_ctas": [_VP, ctypes.c_int32]}.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fp_last_error.argtypes = [_VP]
        L.fp_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor (host or device)
        assert a.is_contiguous()
        return _VP(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return _VP(a.ctypes.data) if a.size else None


def _check(rc, handle=None):
    if rc != FP_OK:
        msg = lib().fp_last_error(handle)
        raise FloodPedError("floodped error %d: %s" % (rc, msg.decode() if msg else ""))


# -- C-ABI entry points, same names ------------------------------------------
def fp_sim_create(cfg: FpConfig):
    h = _VP()
    _check(lib().fp_sim_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def fp_set_stream(h, stream_ptr):
    _check(lib().fp_set_stream(h, _VP(stream_ptr) if stream_ptr else None), h)


def fp_set_terrain(h, z, n0, walkable, exit_mask):
    _check(lib().fp_set_terrain(h, _ptr(z), _ptr(n0), _ptr(walkable), _ptr(exit_mask)), h)


def fp_set_bed(h, z):
    _check(lib().fp_set_bed(h, _ptr(z)), h)


def fp_set_boundary(h, edge, codes):
    _check(lib().fp_set_boundary(h, edge, _ptr(codes)), h)


def fp_set_hydrograph(h, t, depth):
    t = np.ascontiguousarray(t, np.float64)
    depth = np.ascontiguousarray(depth, np.float64)
    _check(lib().fp_set_hydrograph(h, _ptr(t), _ptr(depth), int(t.size)), h)


def fp_set_discharge(h, t, q, h_inflow):
    t = np.ascontiguousarray(t, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    _check(lib().fp_set_discharge(h, _ptr(t), _ptr(q), int(t.size), float(h_inflow)), h)


def fp_set_goals(h, depot, barrier, n_layers):
    depot = np.ascontiguousarray(depot, np.int32)
    barrier = np.ascontiguousarray(barrier, np.int32)
    _check(lib().fp_set_goals(h, _ptr(depot), depot.size, _ptr(barrier), barrier.size, int(n_layers)), h)


def fp_set_doors(h, cells, door, n_doors, entry_period_s, v0_min, v0_max):
    cells = np.ascontiguousarray(cells, np.int32)
    door = np.ascontiguousarray(door, np.int32)
    _check(lib().fp_set_doors(h, _ptr(cells), _ptr(door), int(cells.size), int(n_doors), float(entry_period_s),
                              float(v0_min), float(v0_max)), h)


def fp_set_state(h, depth, hu, hv):
    _check(lib().fp_set_state(h, _ptr(depth), _ptr(hu), _ptr(hv)), h)


def fp_set_time(h, t_ticks, step):
    _check(lib().fp_set_time(h, int(t_ticks), int(step)), h)


def fp_set_barrier_progress(h, total_bags, applied_layers):
    _check(lib().fp_set_barrier_progress(h, int(total_bags), int(applied_layers)), h)


def fp_add_pedestrians(h, recs):
    n = int(recs.shape[0]) if hasattr(recs, "shape") else len(recs)
    _check(lib().fp_add_pedestrians(h, _ptr(recs), n), h)


def fp_clear_pedestrians(h):
    _check(lib().fp_clear_pedestrians(h), h)


def fp_step(h, n):
    _check(lib().fp_step(h, int(n)), h)


def fp_set_step_mode(h, mode):
    _check(lib().fp_set_step_mode(h, int(mode)), h)


def fp_set_tuning(h, tile_rows, ped_lanes):
    _check(lib().fp_set_tuning(h, int(tile_rows), int(ped_lanes)), h)


def fp_set_hash_ahead(h, on):
    _check(lib().fp_set_hash_ahead(h, 1 if on else 0), h)


def fp_set_profiling(h, on):
    _check(lib().fp_set_profiling(h, 1 if on else 0), h)


def fp_synchronize(h):
    _check(lib().fp_synchronize(h), h)


def fp_set_barrier_wait_limit(h, polls):
    _check(lib().fp_set_barrier_wait_limit(h, int(polls)), h)


def fp_read_state(h, which, dst):
    nbytes = dst.numel() * dst.element_size() if hasattr(dst, "data_ptr") else dst.nbytes
    _check(lib().fp_read_state(h, int(which), _ptr(dst), nbytes), h)
    return dst


def fp_water_volume_noalloc(depth, nx, ny, row_pitch, dx, out, stream_ptr=None):
    """Water volume of a caller's device depth grid into a caller's device double; allocates nothing."""
    _check(lib().fp_water_volume_noalloc(_ptr(depth), int(nx), int(ny), int(row_pitch), float(dx), _ptr(out),
                                         _VP(stream_ptr) if stream_ptr else None))


def fp_destroy(h):
    _check(lib().fp_destroy(h))


# -- convenience wrapper ------------------------------------------------------
def ped_records(peds: dict) -> np.ndarray:
    n = int(peds["x"].shape[0])
    r = np.zeros(n, PED_DTYPE)
    for k_src, k_dst in (("x", "x"), ("y", "y"), ("vx", "vx"), ("vy", "vy"), ("role", "role"),
                         ("fsm", "task"), ("timer", "timer_ticks"), ("v0", "v0")):
        r[k_dst] = peds[k_src]
    return r


class Simulation:
    """One simulation handle; methods call the C ABI one to one."""

    def __init__(self, cfg: FpConfig):
        self.cfg = cfg
        self.h = fp_sim_create(cfg)
        self.nx, self.ny = cfg.nx, cfg.ny

    def close(self):
        if self.h is not None:
            fp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        fp_step(self.h, n)

    def synchronize(self):
        fp_synchronize(self.h)

    def add_pedestrians(self, recs):
        fp_add_pedestrians(self.h, recs)

    def field(self, which):
        out = np.empty((self.ny, self.nx), np.float32)
        return fp_read_state(self.h, which, out)

    def peds(self):
        """Every pedestrian so far by id (present or gone)."""
        n = int(self.counters()["n_ids"])
        out = np.zeros(n, PED_DTYPE)
        if n:
            fp_read_state(self.h, FP_FIELD_PEDS, out)
        return out

    def counters(self) -> dict:
        c = FpCounters()
        _check(lib().fp_read_state(self.h, FP_FIELD_COUNTERS, ctypes.byref(c), ctypes.sizeof(c)), self.h)
        return dict(t_ticks=c.t_ticks, step=c.step, n_active=c.n_active, n_exited=c.n_exited,
                    total_bags=c.total_bags, applied_layers=c.applied_layers, neg_depth=c.neg_depth,
                    hist=list(c.hist), wet=c.wet, error_flags=c.error_flags, ped_updates=c.ped_updates,
                    cfl_exceeded=c.cfl_exceeded, n_ids=c.n_ids, n_entered=c.n_entered, n_left=c.n_left)

    def set_fixed_dt(self, dt_seconds):
        _check(lib().fp_set_fixed_dt(self.h, float(dt_seconds)), self.h)

    def surrogate_advance(self, sur, n_windows, mass_tol=1e-4, check_tol=0.01, check_every=8, suspend_windows=8,
                          fix_tol=0.0, stats=None):
        """n_windows windows of 8 fixed steps with the surrogate for the flood update;
        returns the accumulated SurStats (pass it back in to keep accumulating).
        fix_tol > 0: accept net tiles up to that mass residual and close each
        accepted tile's mass balance exactly."""
        g = SurGuard(float(mass_tol), float(check_tol), int(check_every), int(suspend_windows), float(fix_tol))
        st = stats if stats is not None else SurStats()
        _check(lib().fp_surrogate_advance(self.h, sur.h, int(n_windows), ctypes.byref(g), ctypes.byref(st)), self.h)
        return st

    def profile(self) -> dict:
        out = np.zeros(7, np.float64)
        fp_read_state(self.h, FP_FIELD_PROFILE, out)
        return dict(steps=out[0], hash_ms=out[1], flood_ms=out[2], ped_chain_ms=out[3], step_ms=out[4],
                    flood_cells=out[5], ped_ms=out[6])

    def nav(self):
        out = np.empty((3, self.ny, self.nx), np.uint8)
        return fp_read_state(self.h, FP_FIELD_NAV, out)

    def max_hr(self) -> float:
        """Largest hazard rating over the cells holding water (FP_FIELD_HR_MAX)."""
        out = np.zeros(1, np.float32)
        fp_read_state(self.h, FP_FIELD_HR_MAX, out)
        return float(out[0])

    def mass(self):
        out = np.zeros(2, np.float64)
        fp_read_state(self.h, FP_FIELD_MASS, out)
        return float(out[0]), float(out[1])


class Batch:
    """Members (``Simulation`` objects) stepped together by the batched kernels
    (mode FP_MODE_KERNELS) or one persistent kernel (FP_MODE_PERSISTENT)."""

    def __init__(self, sims, mode=None):
        self.sims = list(sims)
        arr = (_VP * len(self.sims))(*[s.h for s in self.sims])
        self.h = _VP()
        _check(lib().fp_batch_create(arr, len(self.sims), ctypes.byref(self.h)))
        if mode is not None:
            self.set_mode(mode)

    def set_mode(self, mode):
        _check(lib().fp_batch_set_step_mode(self.h, int(mode)))

    def step(self, n=1):
        _check(lib().fp_batch_step(self.h, int(n)))

    def synchronize(self):
        _check(lib().fp_batch_synchronize(self.h))

    def close(self):
        if self.h is not None:
            _check(lib().fp_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def config_for(sc, max_peds=None, tile_rows=0) -> FpConfig:
    c = FpConfig()
    c.nx, c.ny, c.dx, c.g, c.cfl = sc.nx, sc.ny, sc.dx, sc.g, sc.cfl
    c.ped_noise, c.t_end, c.seed = sc.ped_noise, sc.t_end, int(sc.seed) & ((1 << 64) - 1)
    c.max_peds = max(sc.n_peds, int(getattr(sc, "max_peds", 0) or 0)) if max_peds is None else max_peds
    c.coupling, c.evac_trigger, c.tile_rows = int(sc.coupling), int(sc.evac_trigger), int(tile_rows)
    c.riemann = int(getattr(sc, "riemann", 0))
    c.order = int(getattr(sc, "order", 1))
    return c


def from_scenario(sc, max_peds=None, tile_rows=0, peds=True, mode=None) -> Simulation:
    """Create a simulation and load a ``scenarios.Scenario`` into it through the C ABI."""
    sim = Simulation(config_for(sc, max_peds, tile_rows))
    if mode is not None:
        fp_set_step_mode(sim.h, mode)
    c = np.ascontiguousarray
    fp_set_terrain(sim.h, c(sc.z, np.float32), c(sc.n0, np.float32), c(sc.walkable, np.uint8),
                   c(sc.exit_mask, np.uint8))
    for edge, codes in ((FP_EDGE_SOUTH, sc.bc_s), (FP_EDGE_NORTH, sc.bc_n), (FP_EDGE_WEST, sc.bc_w),
                        (FP_EDGE_EAST, sc.bc_e)):
        fp_set_boundary(sim.h, edge, c(codes, np.uint8))
    fp_set_hydrograph(sim.h, sc.hydro_t, sc.hydro_h)
    if getattr(sc, "q_t", None) is not None and len(sc.q_t):
        fp_set_discharge(sim.h, sc.q_t, sc.q_Q, sc.h_qin)
    fp_set_goals(sim.h, sc.depot_cells, sc.barrier_cells, sc.n_layers)
    if getattr(sc, "n_doors", 0):
        fp_set_doors(sim.h, sc.door_cells, sc.door_of, sc.n_doors, sc.entry_period, sc.entry_v0[0], sc.entry_v0[1])
    fp_set_state(sim.h, c(sc.h, np.float32), c(sc.hu, np.float32), c(sc.hv, np.float32))
    if getattr(sc, "t0_ticks", 0) or getattr(sc, "step0", 0):
        fp_set_time(sim.h, sc.t0_ticks, sc.step0)
    if getattr(sc, "bags0", 0) or getattr(sc, "applied0", 0):
        fp_set_barrier_progress(sim.h, sc.bags0, sc.applied0)
    if getattr(sc, "dt_fixed_ticks", 0):
        sim.set_fixed_dt(sc.dt_fixed_ticks / TICKS)
    if peds and sc.n_peds:
        sim.add_pedestrians(ped_records(sc.peds))
    return sim


SUR_TILE = 246  # FP_SUR_TILE: output cells per surrogate tile side (256 x 256 net input)


class Surrogate:
    """The learned flood surrogate (tcgen05 forward); parameters as FP32 numpy."""

    CH = (8, 32, 32, 32, 32, 3)  # input: (h, hu, hv, z) as BF16 values, then their BF16 remainders

    def __init__(self, seed=0):
        self.h = _VP()
        _check(lib().fp_surrogate_create(int(seed), ctypes.byref(self.h)))
        self.n_params = lib().fp_surrogate_num_params()

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        _check(lib().fp_surrogate_get_params(self.h, _ptr(out), out.size))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(lib().fp_surrogate_set_params(self.h, _ptr(p), p.size))

    def layers(self, p=None):
        """Split a flat parameter vector into per-layer (w[3,3,ci,co], b[co])."""
        p = self.params() if p is None else p
        out, o = [], 0
        for ci, co in zip(self.CH[:-1], self.CH[1:]):
            w = p[o:o + 9 * ci * co].reshape(3, 3, ci, co)
            o += 9 * ci * co
            b = p[o:o + co]
            o += co
            out.append((w, b))
        return out

    def forward(self, x, y):
        """x: CUDA tensor [B,H,W,4] float32; y: CUDA tensor [B,H-10,W-10,3] float32."""
        B, H, W, _ = x.shape
        _check(lib().fp_surrogate_forward(self.h, _ptr(x), B, H, W, _ptr(y)))
        return y

    def gradients(self, x, target):
        B, H, W, _ = x.shape
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_double()
        _check(lib().fp_surrogate_gradients(self.h, _ptr(x), _ptr(target), B, H, W, _ptr(g), ctypes.byref(loss)))
        return float(loss.value), g

    def train_step(self, x, target, lr):
        B, H, W, _ = x.shape
        loss = ctypes.c_double()
        _check(lib().fp_surrogate_train_step(self.h, _ptr(x), _ptr(target), B, H, W, float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def set_max_ctas(self, ctas):
        """At most ctas CTAs per kernel of the net (0: no limit)."""
        _check(lib().fp_surrogate_set_max_ctas(self.h, int(ctas)))

    @classmethod
    def pretrained(cls, name="shopping_dt1_32"):
        """The net with the parameters shipped in the package's weights folder."""
        sur = cls()
        sur.set_params(np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", name + ".npy")))
        return sur

    def close(self):
        if self.h is not None:
            _check(lib().fp_surrogate_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
