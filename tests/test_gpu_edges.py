"""Degenerate and boundary cases of the coupled step through the C ABI:
one-cell-wide grids, steps past t_end, no pedestrians, capacity and argument
errors, and reading state before any step."""
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


def fields(sim):
    return [sim.field(k) for k in (0, 1, 2)]


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (53, 1), (2, 2), (65, 17)])
def test_thin_grids_match_oracle(P, O, shape):
    nx, ny = shape
    sc = S.random_wet_state(nx, ny, dx=0.7, seed=nx * 31 + ny)
    o = O.Oracle(sc)
    o.step(30)
    sim = P.from_scenario(sc)
    sim.step(30)
    sim.synchronize()
    assert abs(sim.counters()["t_ticks"] - o.t_ticks) <= 30
    for a, b in zip(fields(sim), [o.field(k) for k in ("h", "hu", "hv")]):
        assert np.abs(a - b).max() <= 1e-4


def test_steps_past_t_end_do_nothing(P, O):
    sc = S.plain_coupled_128(seed=3, n_peds=64)
    sc.t_end = 2.0
    o = O.Oracle(sc)
    o.step(10000)
    sim = P.from_scenario(sc)
    sim.step(5000)
    sim.synchronize()
    c = sim.counters()
    assert c["t_ticks"] == o.t_ticks == 2 * 2 ** 20
    before = [f.copy() for f in fields(sim)]
    peds = sim.peds().tobytes()
    sim.step(100)
    sim.synchronize()
    c2 = sim.counters()
    assert c2["t_ticks"] == c["t_ticks"] and c2["step"] == c["step"]
    for a, b in zip(before, fields(sim)):
        assert np.array_equal(a, b)
    assert sim.peds().tobytes() == peds


def test_no_pedestrians_and_zero_steps(P):
    sc = S.plain_coupled_128(seed=4, n_peds=0)
    sim = P.from_scenario(sc)
    h0 = sim.field(0).copy()
    sim.step(0)
    sim.synchronize()
    assert np.array_equal(h0, sim.field(0))
    c = sim.counters()
    assert c["n_active"] == 0 and c["t_ticks"] == 0 and c["step"] == 0
    sim.add_pedestrians(P.ped_records(S.empty_peds(0)))
    sim.step(20)
    sim.synchronize()
    assert sim.counters()["step"] == 20


def test_capacity_and_argument_errors(P):
    sc = S.plain_coupled_128(seed=5, n_peds=10)
    sim = P.from_scenario(sc, max_peds=12)
    recs = P.ped_records(sc.peds)
    with pytest.raises(P.FloodPedError):
        sim.add_pedestrians(recs)  # 10 + 10 > 12
    with pytest.raises(P.FloodPedError):
        sim.step(-1)
    with pytest.raises(P.FloodPedError):
        sim.set_fixed_dt(2.0)
    from paper_1908_05232_b300 import _native as N
    with pytest.raises(P.FloodPedError):  # the C entry point itself (the binding passes 0 or 1)
        N._check(N.lib().fp_set_hash_ahead(sim.h, 2), sim.h)
    with pytest.raises(P.FloodPedError):
        N.fp_set_tuning(sim.h, 12, 8)
    cfg = P.config_for(sc)
    cfg.nx = 0
    with pytest.raises(P.FloodPedError):
        P.Simulation(cfg)
    cfg = P.config_for(sc)
    cfg.tile_rows = 12
    with pytest.raises(P.FloodPedError):
        P.Simulation(cfg)
    # the simulation stays usable after rejected calls
    sim.step(5)
    sim.synchronize()
    assert sim.counters()["step"] == 5


def test_pedestrian_outside_walkable_cells_rejected(P):
    sc = S.plain_coupled_128(seed=6, n_peds=3)
    sim = P.from_scenario(sc, peds=False)
    recs = P.ped_records(sc.peds)
    recs["x"][0] = 0.5 * sc.dx  # the west wall column
    with pytest.raises(P.FloodPedError):
        sim.add_pedestrians(recs)


@pytest.mark.parametrize("mode", ["kernels", "persistent"])
def test_dry_tiles_skipped_after_two_steps(P, mode):
    """A dry domain (walls, no inflow): the first two steps after the state is
    set compute every cell, later steps none (the clock advances apart from the
    cells); the profile counts the computed cell updates."""
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=2, n_peds=64)
    sc.bc_s[:] = S.BC_WALL
    sc.evac_trigger = 0
    m = N.FP_MODE_PERSISTENT if mode == "persistent" else N.FP_MODE_KERNELS
    sim = P.from_scenario(sc, mode=m)
    N.fp_set_profiling(sim.h, 1)
    sim.step(10)
    prof = sim.profile()
    N.fp_set_profiling(sim.h, 0)
    assert prof["steps"] == 10
    assert prof["flood_cells"] == 2 * sc.nx * sc.ny
    assert sim.counters()["t_ticks"] == 10 << 20  # ten dry 1 s steps
    assert all(np.all(f == 0) for f in fields(sim))
    assert sim.counters()["error_flags"] == 0


@pytest.mark.parametrize("mode", ["kernels", "persistent"])
def test_profiled_steps_keep_results(P, mode):
    """Steps in profiling mode (captured with events between the kernels, no
    programmatic launches) give the bytes of unprofiled steps, and the profile
    accounts for every one of them."""
    from paper_1908_05232_b300 import _native as N
    m = N.FP_MODE_KERNELS if mode == "kernels" else N.FP_MODE_PERSISTENT
    sc = S.plain_coupled_128(seed=8)
    a = P.from_scenario(sc, mode=m)
    a.step(30)
    N.fp_set_profiling(a.h, 1)
    a.step(70)
    prof = a.profile()
    N.fp_set_profiling(a.h, 0)
    a.step(20)
    a.synchronize()
    b = P.from_scenario(sc, mode=m)
    b.step(120)
    b.synchronize()
    assert prof["steps"] == 70 and prof["step_ms"] > 0.0
    for k in (0, 1, 2):
        assert np.array_equal(a.field(k), b.field(k))
    assert np.array_equal(a.peds(), b.peds())
