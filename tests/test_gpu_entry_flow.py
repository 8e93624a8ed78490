"""The entry/exit flow through the doors (Sections 2.4, 3 and 3.2) on the GPU
through the C ABI, against the FP64 oracle: visitors admitted per door at each
whole multiple of the entry period, bound for a door drawn with equal
probability, leaving through it, and no admissions once water is seen.

Integers (ids issued, admissions, departures, exits, every record's task,
hazard state and exit byte) must be identical at every step; positions within
1e-3 m (the free-run bound); a visitor's entry position and walking speed are
computed with the same FP32 operations on both sides and must be equal.

Visitors crossing in the corridors come within the 1 m neighbour radius of
one another, where the repulsion's gradient (about 7 m/s^2 per metre at half
a metre) multiplies a position difference several times per 1 s step: FP32
against FP64 rounding then grows past 1e-3 m within tens of steps (seen: 1.8
mm at step 71, 1.4 mm 16 steps after a restart).  The long runs therefore go
in segments from identical inputs: both sides restart from the oracle's state
(FP32-rounded, present pedestrians renumbered in id order) every 25 steps, and
earlier where a position first differs by more than 1e-3 m -- that step is
reported, and it must be a contact: at most three pedestrians, each within
the neighbour radius of another one at that step or the one before.  Every
integer must agree at every step compared."""
import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu
TICKS = 1 << 20


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


def _empty_centre(period=6.0, n=64, dx=5.0, t_end=600.0, capacity=None, seed=3):
    sc = S.shopping_centre(n, dx, 0, 0, seed, t_end, hydro=([0.0], [0.0]))
    return S.with_doors(sc, 7, period, capacity=capacity)


def _flow(c):
    return {k: int(c[k]) for k in ("n_ids", "n_entered", "n_left", "n_exited", "n_active")}


def _compare(sim, o, step, pos_tol=1e-3):
    """Identical integers; returns the records and the ids whose positions
    differ by more than pos_tol."""
    c, fc = sim.counters(), o.flow_counts()
    got = _flow(c)
    want = {k: fc[k] for k in got}
    assert got == want, (step, got, want)
    g, r = sim.peds(), o.peds()
    assert g.shape[0] == r["x"].shape[0]
    assert np.array_equal(g["id"], np.arange(g.shape[0]))
    assert np.array_equal(g["exited"], r["exited"]), step
    assert np.array_equal(g["task"], r["fsm"]), step
    assert np.array_equal(g["hr"], r["hr"]), step
    assert np.array_equal(g["v0"], r["v0"].astype(np.float32)), step
    dpos = np.maximum(np.abs(g["x"] - r["x"]), np.abs(g["y"] - r["y"]))
    return g, r, np.flatnonzero(dpos > pos_tol)


def _in_contact(r, prev, ids, radius=1.0):
    """Each id has another present pedestrian within the radius (now or in
    the previous state)."""
    for st in (r, prev):
        live = np.flatnonzero(st["exited"][: st["x"].shape[0]] == 0)
        ok = True
        for i in ids:
            if i >= st["x"].shape[0]:
                continue
            d = np.hypot(st["x"][live] - st["x"][i], st["y"][live] - st["y"][i])
            d = d[live != i]
            ok &= bool(d.size) and float(d.min()) < radius
        if ok:
            return True
    return False


def _segments(P, O, sc, total_steps, seg_len=25, each_step=None):
    """Lock steps from sc in segments (see the module docstring) until
    total_steps have been compared; returns the summed admissions and
    departures, the divergences (step, ids), the last scenario and oracle."""
    entered = left = done = 0
    divergences = []
    while done < total_steps:
        o = O.Oracle(sc)
        sim = P.from_scenario(sc)
        seen = sim.counters()["n_ids"]
        prev = o.peds()
        for s in range(1, min(seg_len, total_steps - done) + 1):
            o.step(1)
            sim.step(1)
            g, r, bad = _compare(sim, o, (done, s))
            # visitors admitted in this step: at rest at the oracle's entry position
            new = np.arange(seen, g.shape[0])
            stay = new[g["exited"][new] == 0]
            assert np.array_equal(g["x"][stay], r["x"][stay].astype(np.float32))
            assert np.array_equal(g["y"][stay], r["y"][stay].astype(np.float32))
            seen = g.shape[0]
            if each_step is not None:
                each_step(sim, o, g)
            if bad.size:
                assert bad.size <= 3 and _in_contact(r, prev, bad), (done + s, bad.tolist())
                divergences.append((done + s, bad.tolist()))
                break
            prev = r
        done += s
        c = sim.counters()
        assert c["error_flags"] == 0
        entered += c["n_entered"]
        left += c["n_left"]
        sim.close()
        sc = o.to_scenario()
    return entered, left, divergences, sc, o


def test_entry_flow_lockstep(P, O):
    """300 s of entry/exit flow in the empty centre (64 x 64 cells of 5 m, 7
    doors, one visitor per door every 6 s) in 12 segments of 25 steps:
    identical counts and records at every step, entry positions equal to the
    oracle's; 7 x 50 admissions in all, and visitors leave."""
    entered, left, div, _, _ = _segments(P, O, _empty_centre(), 300)
    print("position divergences (step, ids):", div)
    assert entered == 7 * 50 and left > 50 and len(div) <= 30


def test_entry_flow_step_modes_give_the_same_bytes(P):
    """Per-step kernels with and without hash-ahead, the persistent kernel and
    a batch of two members: the same records and counters after 150 steps."""
    from paper_1908_05232_b300 import _native as N
    sc = _empty_centre(period=2.0)
    runs = []
    for mode, ahead in ((N.FP_MODE_KERNELS, 1), (N.FP_MODE_KERNELS, 0), (N.FP_MODE_PERSISTENT, 1)):
        sim = P.from_scenario(sc, mode=mode)
        N.fp_set_hash_ahead(sim.h, ahead)
        sim.step(150)
        sim.synchronize()
        runs.append((sim.peds(), _flow(sim.counters())))
    a, b = P.from_scenario(sc), P.from_scenario(sc)
    batch = P.Batch([a, b])
    batch.step(150)
    batch.synchronize()
    runs += [(a.peds(), _flow(a.counters())), (b.peds(), _flow(b.counters()))]
    batch.close()
    assert runs[0][1]["n_entered"] == 7 * 75
    for peds, flow in runs[1:]:
        assert flow == runs[0][1]
        assert np.array_equal(peds, runs[0][0])


def test_first_water_stops_entries_gpu(P, O):
    """The paper's Scenario 1 at a reduced size (64 x 64 cells of 5.19 m, a
    60 s pre-flood spread, one visitor per door every 2 s, then the
    (160 m^3/s, 7.5 min) discharge flood): in lock step with the oracle through
    the trigger; afterwards no admissions and every visitor is an evacuee."""
    sc = S.scenario1(n=64, dx=5.19, pre_flood=60.0, period=2.0, t_end=400.0)
    # the library's wet flag covers the state a step leaves (the next step
    # sees it); the oracle's is set when a step reads its input state
    state = dict(wet_step=None, step=0, t_wet=None)

    def each_step(sim, o, g):
        state["step"] += 1
        c = sim.counters()
        assert abs(c["t_ticks"] - o.t_ticks) <= 100
        if state["wet_step"] is not None and state["step"] > state["wet_step"]:
            live = g["exited"] == 0
            assert np.all(g["task"][live] == 0)
        if c["wet"] and state["wet_step"] is None:
            state["wet_step"], state["t_wet"] = state["step"], c["t_ticks"]

    entered, left, div, sc_end, o = _segments(P, O, sc, 300, 25, each_step)
    print("position divergences (step, ids):", div)
    assert len(div) <= 30
    # no admission in or after the first wet step: 7 for each whole 2 s before
    # that step's start
    assert state["t_wet"] is not None and state["t_wet"] >= 60 * TICKS
    assert entered == 7 * (state["t_wet"] // (2 * TICKS)) and left > 0
    # the flood from the last segment's end state (water and evacuees in it):
    # one coupled step (identical occupancy on both sides) within the one-step
    # bound, and 20 steps without the roughness coupling within the free-run
    # bound.  Over many coupled steps an evacuee whose position differs by
    # less than the 1e-3 m tolerance can stand in the neighbouring cell on the
    # other side, doubling the Manning n of two cells there: both sides are
    # right for their own positions, and the depths there part by millimetres.
    for coupling, steps, atol, rtol in ((1, 1, 2e-5, 2e-6), (0, 20, 1e-4, 0.0)):
        sc_end.coupling = coupling
        sim = P.from_scenario(sc_end)
        o2 = O.Oracle(sc_end)
        sim.step(steps)
        o2.step(steps)
        assert o2.field("h").max() > 0.3 and o2.counters()["n_active"] > 0
        for k, name in ((0, "h"), (1, "hu"), (2, "hv")):
            ref = o2.field(name)
            err = np.abs(sim.field(k).astype(np.float64) - ref)
            assert np.all(err <= atol + rtol * np.abs(ref)), (coupling, name, err.max())
        sim.close()


def test_lone_visitor_leaves_at_the_oracle_step(P, O):
    """Visitor records added through fp_add_pedestrians (task 8 + door): the
    corridor walk of the oracle pin, on the GPU."""
    nx, ny = 40, 3
    sc = S._base("corridor", nx, ny, 1.0, 1e6, 5)
    sc.walkable[:] = 0
    sc.walkable[1, :] = 1
    sc.z[sc.walkable == 0] = 2.0
    sc.door_cells = np.array([nx, 2 * nx - 1], np.int32)
    sc.door_of = np.array([0, 1], np.int32)
    sc.n_doors, sc.entry_period, sc.evac_trigger, sc.ped_noise = 2, 1e5, 1, 0.0
    p = S.empty_peds(2)
    p["x"][:] = [20.5, 0.5]
    p["y"][:] = 1.5
    p["v0"][:] = 1.2
    p["fsm"][:] = [9, 8]
    sc.peds = p
    o = O.Oracle(sc)
    sim = P.from_scenario(sc)
    for s in range(1, 20):
        o.step(1)
        sim.step(1)
        assert _compare(sim, o, s, pos_tol=1e-4)[2].size == 0  # FP32 positions near 40 m: ulp 4e-6
    g = sim.peds()
    assert list(g["exited"]) == [2, 2] and sim.counters()["n_left"] == 2


def test_capacity_refusal_and_door_validation(P):
    from paper_1908_05232_b300 import _native as N
    sc = _empty_centre(capacity=5)
    sim = P.from_scenario(sc)
    sim.step(30)
    with pytest.raises(N.FloodPedError, match="capacity"):
        sim.synchronize()
    c = sim.counters()
    assert c["n_ids"] == 5 and c["n_entered"] == 5
    sim.step(10)  # the handle stays usable; the admissions at 36 s are refused again
    with pytest.raises(N.FloodPedError):
        sim.synchronize()
    sim.close()
    sc = _empty_centre()
    sim = P.from_scenario(sc)
    wall = int(np.flatnonzero(sc.walkable.reshape(-1) == 0)[0])
    bad = [([wall], [0], 1, 6.0, 1.0, 1.6), ([sc.door_cells[0]], [1], 2, 6.0, 1.0, 1.6),
           ([sc.door_cells[0]], [0], 1, 0.0, 1.0, 1.6), ([sc.door_cells[0]], [0], 1, 6.0, 1.6, 1.0),
           ([sc.door_cells[0]], [0], 9, 6.0, 1.0, 1.6)]
    for cells, door, nd, per, lo, hi in bad:
        with pytest.raises(N.FloodPedError):
            N.fp_set_doors(sim.h, cells, door, nd, per, lo, hi)
    # the terrain resets the doors: nobody enters afterwards
    N.fp_set_terrain(sim.h, sc.z, sc.n0, sc.walkable, sc.exit_mask)
    sim.step(20)
    sim.synchronize()
    assert sim.counters()["n_ids"] == 0
    sim.close()
