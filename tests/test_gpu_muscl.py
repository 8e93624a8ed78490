"""The second-order update (fp_config.order = 2: MUSCL reconstruction, the
centred bed-slope term, two-stage Runge-Kutta) on the GPU through the C ABI,
against the FP64 oracle's: one step and a fixed-step free run of random wet
states with every boundary type (HLL and HLLC, and with discharge breaches),
the coupled plain workload with evacuees raising the roughness, exact lake at
rest and mirror symmetry, the mass balance, the Stoker dam break closer to its
closed form than the first-order update, and the step modes it refuses.
Tolerances as in test_gpu_parity: one step 2e-5 m (+2e-6 relative), free
runs 1e-4 m."""
import math

import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_05232_b300 as pkg
    pkg.build.build()
    return pkg


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


def _fields(sim):
    return [sim.field(k) for k in (0, 1, 2)]


def _close(sim, o, atol, rtol=0.0):
    for a, name in zip(_fields(sim), ("h", "hu", "hv")):
        b = o.field(name)
        err = np.abs(a.astype(np.float64) - b)
        assert np.all(err <= atol + rtol * np.abs(b)), (name, err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("shape,riemann,breach", [((150, 70), 0, False), ((67, 131), 1, False), ((5, 3), 0, False),
                                                  ((96, 40), 0, True)])
def test_one_step_and_free_run(P, O, shape, riemann, breach):
    nx, ny = shape
    sc = S.random_wet_state(nx, ny, dx=0.5, seed=nx * ny + riemann, bc=(2, 1, 0, 1))
    if breach:
        S.with_discharge_breach(sc, "south", nx // 5, nx // 3, 12.0, 80.0, h_inflow=0.8)
        sc.bc_w[ny // 4: ny // 4 + ny // 3] = S.BC_DISCHARGE
        sc.t0_ticks = 10 << 20
    sc.riemann, sc.order = riemann, 2
    o = O.Oracle(sc)
    o.step(1)
    sim = P.from_scenario(sc)
    sim.step(1)
    sim.synchronize()
    assert sim.counters()["t_ticks"] == o.t_ticks
    _close(sim, o, 2e-5, 2e-6)
    sc.dt_fixed_ticks = 1 << 14
    o = O.Oracle(sc)
    o.step(200)
    sim = P.from_scenario(sc)
    sim.step(200)
    sim.synchronize()
    c = sim.counters()
    assert c["t_ticks"] == o.t_ticks and c["neg_depth"] == o.counters()["neg_depth"]
    _close(sim, o, 1e-4)
    m, q = sim.mass()
    assert math.isclose(q, o.boundary_inflow(), rel_tol=1e-5, abs_tol=1e-6)
    assert math.isclose(m, o.mass(), rel_tol=1e-5)


def test_coupled_workload_one_step_and_free_run(P, O):
    """The plain coupled workload (inflow, 256 evacuees whose counts raise the
    Manning n): one step, then 100 steps on a fixed 1/16 s step, the flood
    fields and every pedestrian integer against the oracle."""
    sc = S.plain_coupled_128(seed=2)
    sc.order = 2
    sc.t0_ticks = 40 << 20  # the inflow ramp under way
    o = O.Oracle(sc)
    sim = P.from_scenario(sc)
    o.step(1)
    sim.step(1)
    _close(sim, o, 2e-5, 2e-6)
    sc.dt_fixed_ticks = 1 << 16
    o = O.Oracle(sc)
    sim = P.from_scenario(sc)
    o.step(100)
    sim.step(100)
    sim.synchronize()
    _close(sim, o, 1e-4)
    g, r = sim.peds(), o.peds()
    assert np.array_equal(g["exited"], r["exited"]) and np.array_equal(g["hr"], r["hr"])


def test_lake_at_rest_and_mirror_exact(P):
    sc = S.closed_basin(150, 70, dx=1.0, seed=3)
    sc.order = 2
    sim = P.from_scenario(sc)
    sim.step(200)
    h, hu, hv = _fields(sim)
    z = sim.field(3)
    wet = sc.h > 0
    assert np.all(hu == 0) and np.all(hv == 0)
    assert np.array_equal((h + z)[wet], (sc.h + sc.z)[wet])
    for riemann in (0, 1):
        sc = S.random_wet_state(133, 77, dx=0.7, seed=21, bc=(2, 1, 0, 1))
        sc.order, sc.riemann = 2, riemann
        for axis in ("x", "y"):
            m = sc.copy()
            if axis == "x":
                for f in ("z", "h", "hu", "hv", "n0"):
                    setattr(m, f, np.ascontiguousarray(getattr(sc, f)[:, ::-1]))
                m.hu = -m.hu
                m.bc_w, m.bc_e = sc.bc_e.copy(), sc.bc_w.copy()
                m.bc_s, m.bc_n = sc.bc_s[::-1].copy(), sc.bc_n[::-1].copy()
                fl, su, sv = (lambda f: f[:, ::-1]), -1, 1
            else:
                for f in ("z", "h", "hu", "hv", "n0"):
                    setattr(m, f, np.ascontiguousarray(getattr(sc, f)[::-1, :]))
                m.hv = -m.hv
                m.bc_s, m.bc_n = sc.bc_n.copy(), sc.bc_s.copy()
                m.bc_w, m.bc_e = sc.bc_w[::-1].copy(), sc.bc_e[::-1].copy()
                fl, su, sv = (lambda f: f[::-1, :]), 1, -1
            a, b = P.from_scenario(sc), P.from_scenario(m)
            a.step(60)
            b.step(60)
            a.synchronize()
            b.synchronize()
            ha, hua, hva = _fields(a)
            hb, hub, hvb = _fields(b)
            assert np.array_equal(ha, fl(hb)), (riemann, axis)
            assert np.array_equal(hua, su * fl(hub)) and np.array_equal(hva, sv * fl(hvb)), (riemann, axis)


def test_stoker_closer_than_first_order(P):
    from tests.test_oracle_pins import _stoker
    g = float(np.float32(9.81))
    errs = {}
    for order in (1, 2):
        nx, L, T = 400, 100.0, 4.0
        dx = L / nx
        sc = S.dam_break_1d(nx=nx, ny=3, dx=dx, h_left=1.0, h_right=0.1, t_end=T)
        sc.order = order
        sim = P.from_scenario(sc)
        while sim.counters()["t_ticks"] < int(T * (1 << 20)):
            sim.step(64)
        xc = (np.arange(nx) + 0.5) * dx - 0.5 * L
        h = sim.field(0).astype(np.float64)
        errs[order] = np.abs(h[1] - _stoker(xc, T, 1.0, 0.1, g)).sum() * dx
    assert errs[2] < 0.7 * errs[1], errs


def test_refused_step_forms(P):
    from paper_1908_05232_b300 import _native as N
    sc = S.random_wet_state(40, 30, dx=0.5, seed=1)
    sc.order = 2
    sim = P.from_scenario(sc)
    with pytest.raises(N.FloodPedError):
        N.fp_set_step_mode(sim.h, N.FP_MODE_PERSISTENT)
    with pytest.raises(N.FloodPedError):
        P.Batch([sim])
    sim.set_fixed_dt(2.0 ** -5)
    sur = P.Surrogate(seed=1)
    with pytest.raises(N.FloodPedError):
        sim.surrogate_advance(sur, 1)
    sur.close()
    bad = N.config_for(sc)
    bad.order = 3
    with pytest.raises(N.FloodPedError):
        N.fp_sim_create(bad)
    sim.close()


def test_mostly_dry_grid_parity(P, O):
    """Second order with water in the west third only, inflow on the east
    edge: tiles whose 3 x 3 tile neighbourhood holds no water are skipped
    (their output written as zeros once), the wet front and the edge tiles
    computed; one step and 120 steps against the oracle."""
    sc = S.random_wet_state(300, 200, dx=0.8, seed=21)
    sc.h[:, 100:] = 0.0
    sc.hu[:, 100:] = 0.0
    sc.hv[:, 100:] = 0.0
    sc.order = 2
    o = O.Oracle(sc)
    o.step(1)
    sim = P.from_scenario(sc)
    sim.step(1)
    sim.synchronize()
    assert sim.counters()["t_ticks"] == o.t_ticks
    _close(sim, o, 2e-5, 2e-6)
    o.step(119)
    sim.step(119)
    sim.synchronize()
    assert abs(sim.counters()["t_ticks"] - o.t_ticks) <= 120
    _close(sim, o, 1e-4)


def test_state_write_reopens_skipped_tiles(P):
    """Second order: after the dry east part's tiles are skipped, water put
    there by a state write from the host makes every tile run again -- the run
    continues exactly as a fresh simulation from that state."""
    import copy
    sc = S.random_wet_state(300, 200, dx=0.8, seed=23, bc=(S.BC_WALL,) * 4)
    sc.h[:, 90:] = 0.0
    sc.hu[:, 90:] = 0.0
    sc.hv[:, 90:] = 0.0
    sc.order = 2
    a = P.from_scenario(sc)
    a.step(40)
    a.synchronize()
    h, hu, hv = _fields(a)
    assert np.all(h[:, 200:] == 0.0)
    h[60:120, 220:280] += 0.5
    P._native.fp_set_state(a.h, h, hu, hv)
    sc2 = copy.deepcopy(sc)
    sc2.h, sc2.hu, sc2.hv = h.copy(), hu.copy(), hv.copy()
    b = P.from_scenario(sc2)
    a.step(60)
    b.step(60)
    a.synchronize()
    b.synchronize()
    for x, y in zip(_fields(a), _fields(b)):
        assert np.array_equal(x, y)
    assert np.any(_fields(a)[0][:, 220:280] != 0.0)
