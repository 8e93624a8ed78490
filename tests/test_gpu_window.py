"""Fixed time step and the surrogate window (FP_SUR_WINDOW fixed steps with the
learned net standing in for the flood update, guarded per tile, plain fallback).

Exact properties: a dry domain's window equals plain stepping (the net is never
run and pedestrians see the same state); a zero net keeps a lake at rest exactly
with no fallback; tiles the guard rejects, and windows run on the plain update,
equal plain stepping bit for bit (the fallback recomputes a tile over a region
grown by the window's domain of dependence)."""
import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu

H, HU, HV = 0, 1, 2
DT = 2 ** -6  # s


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


def fields(sim):
    return [sim.field(k) for k in (H, HU, HV)]


def net(P, scale=None, seed=5):
    sur = P.Surrogate(seed=seed)
    if scale is not None:
        p = sur.params()
        sur.set_params(p * np.float32(scale))
    return sur


def fixed(sc, dt=DT):
    sc.dt_fixed_ticks = int(round(dt * 2 ** 20))
    return sc


def test_fixed_dt_parity(P, O):
    sc = fixed(S.random_wet_state(150, 70, dx=0.8, seed=3))
    o = O.Oracle(sc)
    o.step(1)
    sim = P.from_scenario(sc)
    sim.step(1)
    sim.synchronize()
    assert sim.counters()["t_ticks"] == o.t_ticks == sc.dt_fixed_ticks
    for a, b in zip(fields(sim), [o.field(k) for k in ("h", "hu", "hv")]):
        assert np.abs(a - b).max() <= 2e-5 + 2e-6 * np.abs(b).max()
    o.step(49)
    sim.step(49)
    sim.synchronize()
    assert sim.counters()["t_ticks"] == o.t_ticks == 50 * sc.dt_fixed_ticks
    for a, b in zip(fields(sim), [o.field(k) for k in ("h", "hu", "hv")]):
        assert np.abs(a - b).max() <= 1e-4


def test_fixed_dt_courant_counter(P):
    sc = S.random_wet_state(96, 64, dx=1.0, seed=4)
    h = sc.h.astype(np.float64)
    wet = h > 1e-6
    u = np.where(wet, np.abs(sc.hu) / np.where(wet, h, 1), 0)
    v = np.where(wet, np.abs(sc.hv) / np.where(wet, h, 1), 0)
    smax = (np.maximum(u, v) + np.sqrt(9.81 * h))[wet].max()
    smax = max(smax, np.sqrt(9.81 * max(sc.hydro_h)))
    dt_ok = 0.25 * sc.cfl * sc.dx / smax
    for dt, over in ((dt_ok, False), (4 * dt_ok, True)):
        sim = P.from_scenario(fixed(sc, dt))
        sim.step(1)
        sim.synchronize()
        c = sim.counters()
        assert (c["cfl_exceeded"] > 0) == over, (dt, c["cfl_exceeded"])


def test_window_needs_fixed_dt(P):
    sim = P.from_scenario(S.random_wet_state(40, 30, seed=1))
    with pytest.raises(P.FloodPedError):
        sim.surrogate_advance(net(P), 1)


def test_window_dry_domain_equals_plain(P):
    sc = S.plain_coupled_128(seed=2, n_peds=256)
    sc.bc_s[:] = S.BC_WALL
    sc.evac_trigger = 0
    fixed(sc, 1.0 / 16)
    a = P.from_scenario(sc)
    b = P.from_scenario(sc)
    st = a.surrogate_advance(net(P), 4, check_every=0)
    b.step(4 * 8)
    b.synchronize()
    assert st.windows == 4 and st.tiles_net == 0 and st.tiles_fallback == 0
    assert a.counters()["t_ticks"] == b.counters()["t_ticks"] == 32 * sc.dt_fixed_ticks
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)
    pa, pb = a.peds(), b.peds()
    assert pa.tobytes() == pb.tobytes()


def test_window_zero_net_keeps_lake_at_rest(P):
    sc = fixed(S.closed_basin(300, 200, dx=1.0, seed=2))
    sim = P.from_scenario(sc)
    before = fields(sim)
    sur = net(P)
    sur.set_params(np.zeros(sur.n_params, np.float32))
    st = sim.surrogate_advance(sur, 3, check_every=0)
    assert st.windows == 3 and st.tiles_net == 3 * 2 and st.tiles_fallback == 0
    assert st.max_residual == 0.0
    for x, y in zip(before, fields(sim)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", [(300, 140), (520, 260)])
def test_window_fallback_equals_plain(P, shape):
    nx, ny = shape
    sc = fixed(S.random_wet_state(nx, ny, dx=0.8, seed=nx + ny))
    a = P.from_scenario(sc)
    b = P.from_scenario(sc)
    st = a.surrogate_advance(net(P, scale=3.0), 2, mass_tol=0.0, check_every=0)
    b.step(16)
    b.synchronize()
    T = P._native.SUR_TILE
    tiles = ((nx + T - 1) // T) * ((ny + T - 1) // T)
    assert st.tiles_net == 2 * tiles and st.tiles_fallback == 2 * tiles
    assert a.counters()["t_ticks"] == b.counters()["t_ticks"]
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)


def test_window_guard_recomputes_only_rejected_tiles(P):
    # a lake at rest in the west tile column and a wave in the east one: the
    # zero net keeps the lake exactly, the wave tile fails and is recomputed
    T = P._native.SUR_TILE
    sc = fixed(S.random_wet_state(2 * T, 200, dx=0.8, seed=9, bc=(S.BC_WALL,) * 4))
    sc.z[:, :T] = np.round(sc.z[:, :T] * 4096) / 4096
    sc.h[:, :T] = np.maximum(0.0, 1.0 - sc.z[:, :T])
    sc.hu[:, :T] = 0.0
    sc.hv[:, :T] = 0.0
    a = P.from_scenario(sc)
    b = P.from_scenario(sc)
    sur = net(P)
    sur.set_params(np.zeros(sur.n_params, np.float32))
    st = a.surrogate_advance(sur, 1, mass_tol=1e-4, check_every=0)
    b.step(8)
    b.synchronize()
    assert st.tiles_net == 2
    fa, fb = fields(a), fields(b)
    # the wave tile is recomputed (the zero net misses the flow through its
    # west edge); the lake tile, kept by the net or recomputed, is the plain
    # result except where the wave's 8 steps reach across x = T
    assert st.tiles_fallback >= 1
    for x, y in zip(fa, fb):
        assert np.array_equal(x[:, T:], y[:, T:])
    for x, y in zip(fa, fb):
        assert np.array_equal(x[:, :T - 8], y[:, :T - 8])


def test_window_checks_and_suspension(P):
    sc = fixed(S.random_wet_state(300, 140, dx=0.8, seed=11))
    a = P.from_scenario(sc)
    b = P.from_scenario(sc)
    sur = net(P)
    sur.set_params(np.zeros(sur.n_params, np.float32))
    # every window checked, the mass bound off so that every net tile is kept;
    # the persistence forecast misses by more than 1e-6 m, so the windows after
    # the first run the plain update
    st = a.surrogate_advance(sur, 3, mass_tol=1e9, check_tol=1e-6, check_every=1, suspend_windows=5)
    b.step(24)
    b.synchronize()
    assert st.windows == 3 and st.checks >= 1 and st.checks_failed >= 1
    assert st.max_check_error > 1e-6
    assert st.tiles_plain == 3 * 2
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)


def test_window_coupled_run_keeps_invariants(P):
    sc = S.shopping_centre(256, 0.5, 2000, 0, 3, 1800.0)
    fixed(sc, 1.0 / 32)
    sim = P.from_scenario(sc)
    st = sim.surrogate_advance(net(P), 10, check_every=4)
    c = sim.counters()
    assert st.windows == 10
    assert c["t_ticks"] == 80 * sc.dt_fixed_ticks
    assert c["n_active"] + c["n_exited"] == 2000
    assert c["error_flags"] == 0
    p = sim.peds()
    live = p["exited"] == 0
    ci = np.floor(p["x"][live] / sc.dx).astype(int)
    cj = np.floor(p["y"][live] / sc.dx).astype(int)
    assert np.all(sc.walkable[cj, ci] == 1)


def test_window_output_then_plain_steps(P):
    """Plain steps after a window (which may put water into tiles that stayed
    dry before it) continue exactly as a fresh simulation from the window's
    end state."""
    import copy
    sc = fixed(S.random_wet_state(300, 140, dx=0.8, seed=13, bc=(S.BC_WALL,) * 4))
    sc.h[:, 120:] = 0.0
    sc.hu[:, 120:] = 0.0
    sc.hv[:, 120:] = 0.0
    a = P.from_scenario(sc)
    a.step(40)
    a.synchronize()
    before = a.field(H)
    st = a.surrogate_advance(net(P), 1, mass_tol=1e9, check_every=0)
    assert st.tiles_net >= 1
    after = fields(a)
    assert np.any((before == 0.0) & (after[H] != 0.0))
    sc2 = copy.deepcopy(sc)
    sc2.h, sc2.hu, sc2.hv = [x.copy() for x in after]
    b = P.from_scenario(sc2)
    a.step(24)
    b.step(24)
    a.synchronize()
    b.synchronize()
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)



def test_window_mass_fix_closes_the_balance(P):
    """With the mass fix every accepted net tile's volume change equals its
    edge-inflow estimate; neighbouring tiles estimate a shared edge from the
    same cells, so in a walled domain the total volume is kept (an untrained
    net alone changes it)."""
    sc = fixed(S.random_wet_state(300, 140, dx=0.8, seed=17, bc=(S.BC_WALL,) * 4))
    a = P.from_scenario(sc)
    b = P.from_scenario(sc)
    v0 = a.mass()[0]
    sa = a.surrogate_advance(net(P), 2, fix_tol=1e9, check_every=0)
    sb = b.surrogate_advance(net(P), 2, mass_tol=1e9, check_every=0)
    assert sa.tiles_net == sb.tiles_net == 2 * 2 and sa.tiles_fallback == sb.tiles_fallback == 0
    va, vb = a.mass()[0], b.mass()[0]
    assert abs(va - v0) <= 1e-6 * v0
    assert abs(vb - v0) > 1e-5 * v0


def test_window_after_hashed_steps_keeps_results(P):
    """Steps whose pedestrian kernel hashed the records ahead, then a window,
    then more steps give the bytes of the same run without hashing ahead."""
    from paper_1908_05232_b300 import _native as N
    sc = fixed(S.plain_coupled_128(seed=6))
    out = []
    for ahead in (True, False):
        sim = P.from_scenario(sc)
        N.fp_set_hash_ahead(sim.h, ahead)
        sim.step(70)
        sim.surrogate_advance(net(P), 2, check_every=0)
        sim.step(20)
        sim.synchronize()
        out.append((fields(sim), sim.peds(), sim.counters()["ped_updates"]))
    for x, y in zip(out[0][0], out[1][0]):
        assert np.array_equal(x, y)
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


def test_guard_residual_matches_oracle(P, O):
    """The guard's per-tile mass residual, restated in the oracle from the
    window's start and end states: a small random net over two tiles of a wet
    domain (every net tile accepted: mass bound off, no check), the largest
    residual the window records against the oracle's over the same tiles."""
    sc = fixed(S.random_wet_state(300, 120, dx=0.5, seed=6, bc=(2, 1, 0, 0)), dt=2 ** -5)
    sc.peds = S.empty_peds(0)
    sim = P.from_scenario(sc)
    start = [f.astype(np.float64) for f in fields(sim)]
    t0 = sim.counters()["t_ticks"]
    sur = net(P, scale=0.05, seed=8)
    st = sim.surrogate_advance(sur, 1, mass_tol=1e9, check_every=0)
    end = [f.astype(np.float64) for f in fields(sim)]
    t1 = sim.counters()["t_ticks"]
    assert st.tiles_net == 2 and st.tiles_fallback == 0 and st.fail_courant == 0
    assert t1 - t0 == 8 * sc.dt_fixed_ticks
    o = O.Oracle(sc)
    T = 246  # FP_SUR_TILE
    res = [o.guard_residual(start, end, x0, min(x0 + T, sc.nx), 0, sc.ny, t0, t1) for x0 in (0, T)]
    assert max(res) > 1e-4  # the random net moves mass: a residual the guard would reject
    assert abs(st.max_residual - max(res)) <= 1e-3 * max(res), (st.max_residual, res)
