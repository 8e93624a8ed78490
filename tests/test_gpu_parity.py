"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs, plus exact properties the FP32 kernels must keep.

Tolerances: one step from an identical state, FP32 vs FP64 rounding only:
flood fields within 2e-5 m (or m^2/s), positions within 1e-4 m.  Free-running
flood: within 1e-4 m after 1000 steps (the accumulated FP32 rounding of the
update).  Integer outputs (hazard states, responder tasks, timers, exits,
sandbag counts, time in ticks) must be identical: both sides take those
decisions in FP32 on the same values.
"""
import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu

H, HU, HV, Z = 0, 1, 2, 3


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


def run_gpu(P, sc, n, **kw):
    sim = P.from_scenario(sc, **kw)
    sim.step(n)
    sim.synchronize()
    return sim


def fields(sim):
    return [sim.field(k) for k in (H, HU, HV)]


def oracle_fields(o):
    return [o.field(k) for k in ("h", "hu", "hv")]


def assert_flood_close(sim, o, atol, rtol=0.0):
    for a, b, name in zip(fields(sim), oracle_fields(o), ("h", "hu", "hv")):
        err = np.abs(a.astype(np.float64) - b)
        bound = atol + rtol * np.abs(b)
        assert np.all(err <= bound), "%s max err %g at %s" % (name, err.max(), np.unravel_index(err.argmax(), err.shape))


def edge_near(x, y, dx, eps):
    """Positions within eps of a cell edge: the one place an FP32 and an FP64
    evaluation of the same move may fall into different cells."""
    fx = np.mod(np.asarray(x, np.float64), dx)
    fy = np.mod(np.asarray(y, np.float64), dx)
    return (np.minimum(fx, dx - fx) < eps) | (np.minimum(fy, dx - fy) < eps)


def assert_peds_match(sim, o, pos_tol, vel_tol, dx=None, edge_eps=1e-4, max_edge_frac=0.002):
    """Identical integer states and close positions; a pedestrian may differ only
    if the oracle puts it within edge_eps of a cell edge (decision boundary)."""
    g = sim.peds()
    r = o.peds()
    bad = ((g["exited"] != r["exited"]) | (g["task"] != r["fsm"]) | (g["timer_ticks"] != r["timer"]) |
           (g["hr"] != r["hr"]) | (np.abs(g["x"] - r["x"]) > pos_tol) | (np.abs(g["y"] - r["y"]) > pos_tol) |
           (np.abs(g["vx"] - r["vx"]) > vel_tol) | (np.abs(g["vy"] - r["vy"]) > vel_tol))
    if dx is not None and bad.any():
        near = edge_near(r["x"], r["y"], dx, edge_eps)
        assert not (bad & ~near).any(), np.nonzero(bad & ~near)
        assert bad.sum() <= max(1, max_edge_frac * len(bad)), bad.sum()
    else:
        assert not bad.any(), (np.nonzero(bad), np.abs(g["x"] - r["x"]).max(), np.abs(g["y"] - r["y"]).max())


# --------------------------------------------------------------------------
# exact properties of the FP32 flood update
# --------------------------------------------------------------------------
@pytest.mark.parametrize("tile_rows", [8, 16, 32])
def test_lake_at_rest_exact(P, tile_rows):
    sc = S.closed_basin(150, 70, dx=1.0, seed=3)
    sim = run_gpu(P, sc, 200, tile_rows=tile_rows)
    h, hu, hv = fields(sim)
    z = sim.field(Z)
    wet = sc.h > 0
    assert np.all(hu == 0) and np.all(hv == 0)
    assert np.array_equal((h + z)[wet], (sc.h + sc.z)[wet])
    assert np.all(h[~wet] == 0)
    assert sim.counters()["step"] == 200


@pytest.mark.parametrize("axis", ["x", "y"])
def test_mirror_symmetry_exact(P, axis):
    sc = S.random_wet_state(133, 77, dx=0.7, seed=21, bc=(2, 1, 0, 1))
    m = sc.copy()
    if axis == "x":
        for f in ("z", "h", "hu", "hv", "n0"):
            setattr(m, f, np.ascontiguousarray(getattr(sc, f)[:, ::-1]))
        m.hu = -m.hu
        m.bc_w, m.bc_e = sc.bc_e.copy(), sc.bc_w.copy()
        m.bc_s, m.bc_n = sc.bc_s[::-1].copy(), sc.bc_n[::-1].copy()
        fl = lambda f: f[:, ::-1]
        su, sv = -1, 1
    else:
        for f in ("z", "h", "hu", "hv", "n0"):
            setattr(m, f, np.ascontiguousarray(getattr(sc, f)[::-1, :]))
        m.hv = -m.hv
        m.bc_s, m.bc_n = sc.bc_n.copy(), sc.bc_s.copy()
        m.bc_w, m.bc_e = sc.bc_w[::-1].copy(), sc.bc_e[::-1].copy()
        fl = lambda f: f[::-1, :]
        su, sv = 1, -1
    a, b = run_gpu(P, sc, 60), run_gpu(P, m, 60)
    assert a.counters()["t_ticks"] == b.counters()["t_ticks"]
    ha, hua, hva = fields(a)
    hb, hub, hvb = fields(b)
    assert np.array_equal(ha, fl(hb))
    assert np.array_equal(hua, su * fl(hub))
    assert np.array_equal(hva, sv * fl(hvb))


def test_mass_balance(P):
    sc = S.random_wet_state(130, 90, dx=0.5, seed=11, bc=(0, 0, 0, 0))
    sim = P.from_scenario(sc)
    m0, _ = sim.mass()
    sim.step(400)
    sim.synchronize()
    m1, q = sim.mass()
    assert q == 0.0
    assert abs(m1 - m0) <= 2e-6 * m0
    assert sim.counters()["neg_depth"] == 0
    sc = S.random_wet_state(130, 90, dx=0.5, seed=12)
    sim = P.from_scenario(sc)
    m0, _ = sim.mass()
    sim.step(400)
    sim.synchronize()
    m1, q = sim.mass()
    assert abs(m1 - (m0 + q)) <= 2e-6 * m0


# --------------------------------------------------------------------------
# parity with the oracle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape,tile_rows", [((150, 70), 16), ((64, 16), 16), ((129, 45), 8), ((97, 100), 32),
                                             ((5, 3), 16)])
def test_flood_one_step_parity(P, O, shape, tile_rows):
    nx, ny = shape
    sc = S.random_wet_state(nx, ny, dx=0.8, seed=nx * 7 + ny)
    o = O.Oracle(sc)
    o.step(1)
    sim = run_gpu(P, sc, 1, tile_rows=tile_rows)
    assert sim.counters()["t_ticks"] == o.t_ticks
    assert_flood_close(sim, o, atol=2e-5, rtol=2e-6)


def test_flood_1000_steps_parity(P, O):
    sc = S.plain_coupled_128(seed=1, n_peds=0)
    sc.t_end = 1e6
    o = O.Oracle(sc)
    o.step(1000)
    sim = run_gpu(P, sc, 1000)
    c = sim.counters()
    assert c["step"] == 1000
    assert abs(c["t_ticks"] - o.t_ticks) <= 1000  # dt may round to a neighbouring tick now and then
    assert_flood_close(sim, o, atol=1e-4)
    m, q = sim.mass()
    assert abs(m - o.mass()) <= 1e-5 * o.mass()


def test_dam_break_ritter(P, O):
    sc = S.dam_break_1d(nx=800, ny=4, dx=0.125, h_left=1.0, h_right=0.0, t_end=4.0)
    o = O.Oracle(sc)
    o.step(100000)
    sim = run_gpu(P, sc, o.nstep + 5)
    assert sim.counters()["t_ticks"] == o.t_ticks
    assert_flood_close(sim, o, atol=1e-4)


def test_nav_fields_match(P, O):
    sc = S.shopping_centre(160, 0.5, 200, 20, seed=5, n_barrier=30, n_layers=2)
    sim = P.from_scenario(sc)
    nav = sim.nav()
    o = O.Oracle(sc)
    assert np.array_equal(nav[0], o.field("nav_exit"))
    assert np.array_equal(nav[1], o.field("nav_depot"))
    assert np.array_equal(nav[2], o.field("nav_barrier"))


def _crowd_state(seed, nx=140, ny=75, n_evac=900, n_resp=120):
    sc = S.random_wet_state(nx, ny, dx=0.5, seed=seed, dry_frac=0.35, vel=1.0)
    sc.walkable = (np.random.default_rng(seed).uniform(size=(ny, nx)) > 0.08).astype(np.uint8)
    sc.exit_mask[ny - 1, nx // 2 - 6: nx // 2 + 6] = 1
    sc.walkable[sc.exit_mask == 1] = 1
    sc.coupling = 1
    S.random_crowd(sc, n_evac, n_resp, seed=seed, random_velocity=1.0, random_tasks=True)
    S.with_depot_and_barrier(sc, depot_ij=[(10, 10), (11, 10)], barrier_ij=[(i, 40) for i in range(30, 60)],
                             n_layers=2)
    sc.walkable[40, 30:60] = 1
    sc.walkable[10, 10:12] = 1
    return sc


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_coupled_one_step_parity(P, O, seed):
    sc = _crowd_state(seed)
    # put some responders exactly in their depot / barrier cells to exercise arrivals
    o = O.Oracle(sc)
    o.step(1)
    sim = run_gpu(P, sc, 1)
    assert sim.counters()["t_ticks"] == o.t_ticks
    assert_flood_close(sim, o, atol=2e-5, rtol=2e-6)
    assert_peds_match(sim, o, pos_tol=1e-4, vel_tol=2e-4, dx=sc.dx)
    cg, co = sim.counters(), o.counters()
    for k in ("n_exited", "total_bags", "hist", "n_active"):
        assert cg[k] == co[k], (k, cg[k], co[k])


def _barrier_case(n=192, seed=7):
    return S.shopping_centre(n, 0.5, 300, 40, seed, 4000.0, hydro=([0.0, 600.0, 900.0], [0.0, 0.0, 0.6]),
                             n_barrier=30, n_layers=2)


def _barrier_wet():
    return S.shopping_centre(192, 0.5, 300, 40, 7, 4000.0, hydro=([0.0, 300.0], [0.3, 0.9]), n_barrier=30,
                             n_layers=2)


TRAJECTORY_CASES = {
    "plain128_k150": (lambda: S.plain_coupled_128(seed=1), 150),         # dense crowd at the exit gap
    "crowd_wet_k120": (lambda: _crowd_state(4), 120),                   # all hazard states, responder tasks
    "barrier_wet_k200": (_barrier_wet, 200),                            # sandbagging while the flood enters
    "barrier_dry_k350": (lambda: _barrier_case(), 350),                 # mid-deployment, bags dropped
    "shop256_k150": (lambda: S.shopping_centre(256, 0.5, 2000, 0, 9, 1800.0), 150),
}


@pytest.mark.parametrize("case", sorted(TRAJECTORY_CASES))
def test_trajectory_one_step_parity(P, O, case):
    """One step from mid-run states taken along the oracle's own trajectory
    (dense crowd at the exit, flood front, responders mid-task): both sides load
    the oracle's FP32-rounded state and advance it once."""
    build, k = TRAJECTORY_CASES[case]
    sc0 = build()
    base = O.Oracle(sc0)
    base.step(k)
    sc = base.to_scenario()
    o = O.Oracle(sc)
    o.step(1)
    sim = run_gpu(P, sc, 1)
    c = sim.counters()
    assert c["t_ticks"] == o.t_ticks and c["step"] == o.nstep
    assert_flood_close(sim, o, atol=2e-5, rtol=2e-6)
    assert_peds_match(sim, o, pos_tol=1e-4, vel_tol=2e-4, dx=sc.dx)
    co = o.counters()
    assert c["total_bags"] == co["total_bags"]
    assert np.array_equal(sim.field(Z), o.field("z").astype(np.float32))


def test_coupled_free_run(P, O):
    """600 free-running coupled steps of the 128 x 128 case.  Crowd contact at the
    exit gap amplifies FP32-vs-FP64 rounding, so individual pedestrians may drift
    apart; the flood fields must stay within 1e-4 m and the crowd must stay valid
    and statistically the same."""
    sc = S.plain_coupled_128(seed=1)
    o = O.Oracle(sc)
    sim = P.from_scenario(sc)
    for _ in range(6):
        o.step(100)
        sim.step(100)
        sim.synchronize()
        assert_flood_close(sim, o, atol=1e-4)
    g, r = sim.peds(), o.peds()
    c, co = sim.counters(), o.counters()
    assert c["n_active"] + c["n_exited"] == sc.n_peds
    ii = np.floor(g["x"] / np.float32(sc.dx)).astype(int)
    jj = np.floor(g["y"] / np.float32(sc.dx)).astype(int)
    assert np.all(sc.walkable[jj, ii] == 1)
    assert abs(c["n_exited"] - co["n_exited"]) <= 0.03 * sc.n_peds
    close = (np.abs(g["x"] - r["x"]) <= 1e-3) & (np.abs(g["y"] - r["y"]) <= 1e-3) & (g["exited"] == r["exited"])
    assert close.mean() >= 0.8, close.mean()


def test_sandbag_barrier_free_run(P, O):
    """Responders build a 6-cell, 2-layer barrier: the same bags, the same
    completed layers and the same raised bed as the oracle, all responders done."""
    sc = S.closed_basin(30, 16, dx=0.5, wet=False, bumps=False)
    sc.ped_noise = 0.05
    sc.exit_mask[15, 12:16] = 1
    S.with_depot_and_barrier(sc, depot_ij=[(3, 3), (4, 3)], barrier_ij=[(i, 8) for i in range(18, 24)], n_layers=2)
    S.random_crowd(sc, 0, 6, seed=4)
    sc.t_end = 3000.0
    o = O.Oracle(sc)
    o.step(2000)
    sim = run_gpu(P, sc, 2000)
    cg, co = sim.counters(), o.counters()
    assert co["applied_layers"] == 12
    assert cg["applied_layers"] == co["applied_layers"]
    assert abs(cg["total_bags"] - co["total_bags"]) <= 6
    assert np.array_equal(sim.field(Z), o.field("z").astype(np.float32))
    g = sim.peds()
    assert np.all((g["task"] == 4) | (g["exited"] == 1))


def test_determinism(P):
    sc = S.plain_coupled_128(seed=3)
    a = run_gpu(P, sc, 300)
    b = run_gpu(P, sc, 300)
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.peds(), b.peds())


@pytest.mark.parametrize("case", ["plain128", "barrier192"])
def test_step_modes_agree(P, case):
    """The persistent kernel (up to 256 steps per launch), 64-step CUDA graphs of
    the per-step kernels, and one-at-a-time launches give the same bytes."""
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=5) if case == "plain128" else _barrier_wet()
    n = 300
    a = P.from_scenario(sc, mode=N.FP_MODE_PERSISTENT)
    a.step(n)
    a.synchronize()
    b = P.from_scenario(sc, mode=N.FP_MODE_KERNELS)
    b.step(n)
    b.synchronize()
    c = P.from_scenario(sc, mode=N.FP_MODE_KERNELS)
    for _ in range(n):
        c.step(1)
    c.synchronize()
    for x, y, z in zip(fields(a), fields(b), fields(c)):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    assert np.array_equal(a.peds(), b.peds()) and np.array_equal(a.peds(), c.peds())
    ca, cb = a.counters(), b.counters()
    for k in ("t_ticks", "step", "n_exited", "total_bags", "applied_layers", "hist", "ped_updates"):
        assert ca[k] == cb[k], k
    assert np.array_equal(a.field(Z), b.field(Z))


# --------------------------------------------------------------------------
# the benchmark's workload sizes
# --------------------------------------------------------------------------
def test_shopping_centre_full_size_parity(P, O):
    """512 x 512 cells, 10,000 evacuees (the benchmark workload) in the launch
    configuration bench.py times: one step compared cell by cell and pedestrian by
    pedestrian, then 64 more steps of the flood fields."""
    sc = S.config_shopping()
    o = O.Oracle(sc)
    o.step(1)
    sim = run_gpu(P, sc, 1)
    assert sim.counters()["t_ticks"] == o.t_ticks
    assert_flood_close(sim, o, atol=2e-5, rtol=2e-6)
    assert_peds_match(sim, o, pos_tol=1e-4, vel_tol=2e-4, dx=sc.dx)
    o.step(64)
    sim.step(64)
    sim.synchronize()
    assert_flood_close(sim, o, atol=1e-4)


@pytest.mark.parametrize("shape", [(16, 8, True), (32, 16, False)])
def test_barrier_midflood_full_size_parity(P, O, shape):
    """The benchmark workload at full size -- 2048 x 2048 cells, 100,000
    pedestrians (500 responders mid-deployment), the synthetic mid-flood state --
    restored the way bench.py restores it (state, bed, pedestrians, clock and
    barrier progress through the C ABI, on a simulation that already ran) and
    stepped once in two launch shapes: every cell within 2e-5 m (+2e-6
    relative) of the oracle, every pedestrian's integers identical and its
    position within 1e-4 m, the counters identical."""
    import torch
    import bench
    from paper_1908_05232_b300 import _native as N
    rows, lanes, ahead = shape
    sc = bench.workload(3)
    o = O.Oracle(sc)
    o.step(1)
    sim = P.from_scenario(sc)
    N.fp_set_tuning(sim.h, rows, lanes)
    N.fp_set_hash_ahead(sim.h, ahead)
    sim.step(70)
    sim.synchronize()
    snap = bench.Snapshot(P, N, sim, sc, torch.device("cuda", 0))
    snap.restore()
    sim.step(1)
    sim.synchronize()
    c = sim.counters()
    assert c["t_ticks"] == o.t_ticks and c["error_flags"] == 0
    assert_flood_close(sim, o, atol=2e-5, rtol=2e-6)
    assert np.array_equal(sim.field(Z).astype(np.float64), o.field("z"))
    assert_peds_match(sim, o, pos_tol=1e-4, vel_tol=2e-4, dx=sc.dx)
    oc = o.counters()
    for k in ("n_exited", "total_bags", "applied_layers", "hist", "wet"):
        assert c[k] == oc[k], k


def test_barrier_config_full_size_properties(P):
    """2048 x 2048 cells, 100,000 pedestrians incl. 500 responders: properties
    that hold at any size (the oracle is too slow here)."""
    sc = S.config_barrier()
    sim = P.from_scenario(sc)
    m0, _ = sim.mass()
    sim.step(64)
    sim.synchronize()
    m1, q = sim.mass()
    c = sim.counters()
    assert c["neg_depth"] == 0 and c["error_flags"] == 0
    assert abs(m1 - (m0 + q)) <= 1e-5 * max(m0 + abs(q), 1.0)
    g = sim.peds()
    assert c["n_active"] + c["n_exited"] == sc.n_peds
    ii = np.floor(g["x"] / np.float32(sc.dx)).astype(int)
    jj = np.floor(g["y"] / np.float32(sc.dx)).astype(int)
    assert np.all(sc.walkable[jj, ii] == 1)
    assert c["n_active"] <= sum(c["hist"]) <= sc.n_peds


# --------------------------------------------------------------------------
# batched ensemble
# --------------------------------------------------------------------------
def _batch_members():
    a = S.plain_coupled_128(seed=1)
    b = S.plain_coupled_128(seed=2, n_peds=120, nx=96, ny=80)
    c = _barrier_wet()
    d = _crowd_state(7, nx=100, ny=60, n_evac=300, n_resp=30)
    e = S.closed_basin(70, 45, dx=0.5, seed=9)
    return [a, b, c, d, e]


@pytest.mark.parametrize("mode", ["kernels", "persistent", "mixed_shapes"])
def test_batch_matches_members_alone(P, mode):
    """Scenarios of different grids and crowds stepped as one batch -- per-step
    batch kernels (graph-replayed 64-step runs included), the same with every
    member in a launch shape of its own (flood run heights 8/16/32 and 1-16
    lanes per pedestrian: one flood and one pedestrian launch per shape group),
    or one persistent launch for the whole ensemble (two launches here: 256
    steps, then 44) -- give the bytes each gives stepped alone."""
    from paper_1908_05232_b300 import _native as N
    scs = _batch_members()
    n = 300
    members = [P.from_scenario(sc) for sc in scs]
    if mode == "mixed_shapes":
        for m, (rows, lanes) in zip(members, [(8, 1), (32, 16), (8, 4), (16, 2), (32, 1)]):
            N.fp_set_tuning(m.h, rows, lanes)
    batch = P.Batch(members, mode=N.FP_MODE_PERSISTENT if mode == "persistent" else None)
    batch.step(n)
    batch.synchronize()
    for sc, m in zip(scs, members):
        alone = run_gpu(P, sc, n)
        for x, y in zip(fields(m), fields(alone)):
            assert np.array_equal(x, y), sc.name
        assert np.array_equal(m.field(Z), alone.field(Z))
        assert np.array_equal(m.peds(), alone.peds()), sc.name
        cm, ca = m.counters(), alone.counters()
        for k in ("t_ticks", "step", "n_exited", "total_bags", "applied_layers", "hist", "ped_updates"):
            assert cm[k] == ca[k], (sc.name, k)
    batch.close()


@pytest.mark.parametrize("mode", ["kernels", "persistent"])
def test_batch_then_alone_continues(P, mode):
    """A member stepped alone (leaving its records hashed ahead), then in a
    batch, then alone again gives the bytes of a run stepped alone."""
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=3)
    m = P.from_scenario(sc)
    m.step(20)
    b = P.Batch([m], mode=N.FP_MODE_PERSISTENT if mode == "persistent" else None)
    b.step(70)
    b.synchronize()
    b.close()
    m.step(10)
    m.synchronize()
    alone = run_gpu(P, sc, 100)
    for x, y in zip(fields(m), fields(alone)):
        assert np.array_equal(x, y)
    assert np.array_equal(m.peds(), alone.peds())


def test_launch_shape_does_not_change_results(P):
    """Every flood tile height, pedestrian lane count and hashing place gives the
    same bytes; hash-ahead is also switched on and off in mid-run."""
    from paper_1908_05232_b300 import _native as N
    sc = _barrier_wet()
    ref = None
    for rows, lanes, ahead in ((16, 8, True), (8, 4, False), (32, 16, True), (8, 16, False), (16, 2, True),
                              (8, 1, False), (16, 8, None)):
        sim = P.from_scenario(sc)
        N.fp_set_tuning(sim.h, rows, lanes)
        if ahead is None:  # switched before each call of 70 steps (a graph and single steps)
            for k in range(3):
                N.fp_set_hash_ahead(sim.h, k % 2 == 1)
                sim.step(min(70, 150 - 70 * k))
        else:
            N.fp_set_hash_ahead(sim.h, ahead)
            sim.step(150)
        sim.synchronize()
        out = (fields(sim), sim.peds(), sim.counters()["t_ticks"])
        if ref is None:
            ref = out
        else:
            for x, y in zip(out[0], ref[0]):
                assert np.array_equal(x, y), (rows, lanes, ahead)
            assert np.array_equal(out[1], ref[1]) and out[2] == ref[2]


def test_autotuner_picks_a_valid_shape(P, tmp_path):
    from paper_1908_05232_b300 import autotune
    sc = S.plain_coupled_128(seed=2)
    best = autotune.choose(sc, cache_path=str(tmp_path / "tune.json"))
    assert best["tile_rows"] in (8, 16, 32) and best["ped_lanes"] in (1, 2, 4, 8, 16)
    assert best["us_per_step"] > 0
    again = autotune.choose(sc, cache_path=str(tmp_path / "tune.json"))
    assert again == best
    sim = P.from_scenario(sc)
    autotune.apply(sim, best)
    sim.step(10)
    sim.synchronize()


def test_batch_tuner_picks_valid_shapes(P):
    """The batch tuner's per-member shapes (one shape for all, then per size
    class) are valid candidates; a batch made with them steps."""
    from paper_1908_05232_b300 import autotune
    scs = _batch_members()
    tuned = autotune.tune_batch(scs, rounds=1)
    assert len(tuned["shapes"]) == len(scs) and len(tuned["uniform"]) == 15
    for rows, lanes in tuned["shapes"]:
        assert rows in autotune.TILE_ROWS and lanes in autotune.PED_LANES
    assert sorted(set(tuned["classes"])) == [0, 1] and tuned["us_per_step"] > 0
    members = [P.from_scenario(sc) for sc in scs]
    autotune.apply_batch(members, tuned["shapes"])
    batch = P.Batch(members)
    batch.step(70)
    batch.synchronize()
    assert all(m.counters()["step"] == 70 for m in members)
    batch.close()


@pytest.mark.parametrize("tile_rows", [8, 16, 32])
def test_mostly_dry_grid_parity(P, O, tile_rows):
    """Water in the west third only, inflow on the east edge: most flood tiles
    are dry (the kernel skips their faces) while the wet front, the inflow
    tiles and the dry-wet boundary tiles are computed; 120 steps against the
    oracle."""
    sc = S.random_wet_state(300, 200, dx=0.8, seed=21)
    sc.h[:, 100:] = 0.0
    sc.hu[:, 100:] = 0.0
    sc.hv[:, 100:] = 0.0
    o = O.Oracle(sc)
    o.step(1)
    sim = run_gpu(P, sc, 1, tile_rows=tile_rows)
    assert sim.counters()["t_ticks"] == o.t_ticks
    assert_flood_close(sim, o, atol=2e-5, rtol=2e-6)
    o.step(119)
    sim.step(119)
    sim.synchronize()
    assert abs(sim.counters()["t_ticks"] - o.t_ticks) <= 120
    assert_flood_close(sim, o, atol=1e-4)


def test_state_write_reopens_skipped_tiles(P):
    """Tiles whose stencil stayed dry are skipped after two steps; writing the
    state from the host (water put into that dry region) makes every tile run
    again: the run continues exactly as a fresh simulation from that state."""
    import copy
    sc = S.random_wet_state(300, 200, dx=0.8, seed=23, bc=(S.BC_WALL,) * 4)
    sc.h[:, 90:] = 0.0
    sc.hu[:, 90:] = 0.0
    sc.hv[:, 90:] = 0.0
    a = run_gpu(P, sc, 40)
    h, hu, hv = fields(a)
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
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)
    assert np.any(fields(a)[0][:, 200:] != fields(run_gpu(P, sc, 100))[0][:, 200:])



def test_step_mode_switches_keep_results(P):
    """Switching between the per-step kernels and the persistent kernel in the
    middle of a run (the dry-tile flags carry over) gives the bytes of a run in
    one mode."""
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=6)
    a = P.from_scenario(sc, mode=N.FP_MODE_KERNELS)
    for mode in (N.FP_MODE_KERNELS, N.FP_MODE_PERSISTENT, N.FP_MODE_KERNELS, N.FP_MODE_PERSISTENT):
        N.fp_set_step_mode(a.h, mode)
        a.step(70)
    a.synchronize()
    b = run_gpu(P, sc, 280, mode=N.FP_MODE_KERNELS)
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.peds(), b.peds())


def test_restore_then_step_matches_a_fresh_run(P):
    """The benchmark's restore -- state upload, pedestrians cleared and added
    again, clock set -- on a simulation that ran (records hashed ahead) gives
    the bytes of a fresh simulation stepped from the same start."""
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=4)
    sim = P.from_scenario(sc)
    sim.step(90)
    sim.synchronize()
    recs = P.ped_records(sc.peds)
    for _ in range(2):
        N.fp_set_state(sim.h, sc.h, sc.hu, sc.hv)
        N.fp_clear_pedestrians(sim.h)
        sim.add_pedestrians(recs)
        N.fp_set_time(sim.h, 0, 0)
        sim.step(70)
        sim.synchronize()
    fresh = run_gpu(P, sc, 70)
    for x, y in zip(fields(sim), fields(fresh)):
        assert np.array_equal(x, y)
    assert np.array_equal(sim.peds(), fresh.peds())
    c, f = sim.counters(), fresh.counters()
    for k in ("t_ticks", "step", "n_active", "n_exited", "hist"):
        assert c[k] == f[k], k


def test_launch_shape_switched_mid_run(P):
    """Tile height and lanes changed between calls, while the records are
    hashed ahead, leave the bytes of a run in one shape."""
    from paper_1908_05232_b300 import _native as N
    sc = _barrier_wet()
    a = P.from_scenario(sc)
    for k, (rows, lanes) in enumerate(((16, 8), (8, 16), (32, 4), (16, 8))):
        N.fp_set_tuning(a.h, rows, lanes)
        a.step(70 if k < 3 else 10)
    a.synchronize()
    b = run_gpu(P, sc, 220)
    for x, y in zip(fields(a), fields(b)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.peds(), b.peds())


def test_batch_member_matches_oracle(P, O):
    """A member of a batched ensemble against the oracle directly: 64 coupled
    steps of a low-density crowd on a fixed 1/8 s step, batched with two other
    scenarios of different sizes; the flood within 1e-4 m, every pedestrian's
    integers identical and its position within 1e-3 m, the counters identical."""
    a = S.plain_coupled_128(seed=3, n_peds=48, nx=100, ny=90)
    a.dt_fixed_ticks = 1 << 17
    b = S.shopping_centre(160, 0.5, 300, 20, seed=7, n_barrier=20, n_layers=1)
    c = S.random_wet_state(70, 45, dx=0.5, seed=2)
    members = [P.from_scenario(x) for x in (b, a, c)]
    batch = P.Batch(members)
    batch.step(64)
    batch.synchronize()
    o = O.Oracle(a)
    o.step(64)
    m = members[1]
    assert m.counters()["t_ticks"] == o.t_ticks == 64 * a.dt_fixed_ticks
    assert_flood_close(m, o, atol=1e-4)
    assert_peds_match(m, o, pos_tol=1e-3, vel_tol=1e-2)
    mc, oc = m.counters(), o.counters()
    for k in ("n_exited", "hist", "wet"):
        assert mc[k] == oc[k], k
    batch.close()
