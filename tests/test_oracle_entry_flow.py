"""Pins of the oracle's entry/exit flow (Sections 2.4, 3 and 3.2: visitors
enter through the entrance doors at a constant rate per door, leave through a
door drawn with equal probability, and stop entering once water is seen, when
everyone present evacuates).  CPU only.

What fixes the values: integer counts in closed form (a door admits one
visitor at each whole multiple of the entry period), the equal door
probabilities (a binomial bound on 70,000 draws), numpy's independent Philox
for the generator block a visitor's draws come from, the geometry of a
straight corridor (arrival step of a lone visitor), and conservation of ids
(every id is present, gone through its door or gone through the exit)."""
import math

import numpy as np
import pytest

import scenarios as S

TICKS = 1 << 20


def _philox_numpy(ctr, key):
    """One Philox4x64-10 block from numpy's own implementation."""
    # numpy increments the 256-bit counter before each block: start one below
    v = (sum(int(w) << (64 * k) for k, w in enumerate(ctr)) - 1) % (1 << 256)
    c = [(v >> (64 * k)) & (2**64 - 1) for k in range(4)]
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def test_visitor_draws_equal_door_probabilities(oracle_mod):
    """70,000 visitors over 7 doors: each door's share within 5 sigma of 1/7
    (Section 3); offsets in [1/4, 3/4) of a cell with mean 1/2; speeds in the
    stated range."""
    n, nd = 70_000, 7
    counts = np.zeros(nd, int)
    offs, v0s = [], []
    for pid in range(n):
        ox, oy, v0, d = oracle_mod.visitor_draw(11, pid, nd, 1.0, 1.6)
        counts[d] += 1
        if pid < 5000:
            offs += [ox, oy]
            v0s.append(v0)
    sigma = math.sqrt(n * (1 / nd) * (1 - 1 / nd))
    assert np.all(np.abs(counts - n / nd) < 5 * sigma), counts
    offs, v0s = np.array(offs), np.array(v0s)
    assert offs.min() >= 0.25 and offs.max() < 0.75
    assert abs(offs.mean() - 0.5) < 0.005
    assert v0s.min() >= np.float32(1.0) and v0s.max() <= np.float32(1.6)
    assert abs(v0s.mean() - 1.3) < 0.01
    # one door: every visitor is bound for it
    assert {oracle_mod.visitor_draw(11, p, 1, 1.0, 1.6)[3] for p in range(200)} == {0}


@pytest.mark.parametrize("pid", [0, 1, 77, 123456])
def test_visitor_draws_come_from_their_own_generator_block(oracle_mod, pid):
    """The draws are the block at counter (id, 0, 1, 0) under the run's seed
    (numpy's Philox), not the per-step block (id, step, 0, 0)."""
    seed = 0xC0FFEE
    r = _philox_numpy([pid, 0, 1, 0], [seed, 0])
    ox, oy, v0, d = oracle_mod.visitor_draw(seed, pid, 7, 1.0, 1.6)
    assert d == ((r[2] >> 40) * 7) >> 24
    assert ox == 0.25 + 0.5 * ((r[0] >> 42) / 2.0**22)
    assert oy == 0.25 + 0.5 * ((r[1] >> 42) / 2.0**22)
    step_block = _philox_numpy([pid, 0, 0, 0], [seed, 0])
    assert d != ((step_block[2] >> 40) * 7) >> 24 or ox != 0.25 + 0.5 * ((step_block[0] >> 42) / 2.0**22)


def _empty_centre(period=6.0, n=64, dx=5.0, t_end=600.0, capacity=None, seed=3):
    sc = S.shopping_centre(n, dx, 0, 0, seed, t_end, hydro=([0.0], [0.0]))
    return S.with_doors(sc, 7, period, capacity=capacity)


@pytest.mark.parametrize("period,dt", [(6.0, 0.0), (2.5, 0.0), (6.0, 0.25)])
def test_entry_counts_closed_form(oracle_mod, period, dt):
    """While dry, each door admits one visitor at each whole multiple of the
    period: after time t, 7 floor(t / period) visitors, ids in order, each
    entering in its door's entry cell (dt = 0: the dry 1 s step)."""
    sc = _empty_centre(period)
    if dt:
        sc.dt_fixed_ticks = int(dt * TICKS)
    o = oracle_mod.Oracle(sc)
    seen = 0
    for _ in range(40):
        o.step(1)
        t = o.t_ticks
        want = 7 * (t // int(period * TICKS))
        fc = o.flow_counts()
        assert fc["n_entered"] == want and fc["n_ids"] == want
        assert fc["n_ids"] == fc["n_active"] + fc["n_left"] + fc["n_exited"]
        p = o.peds()
        # the new ids, door by door: entry positions inside that door's cell
        # (a visitor bound for its entry door may already have left)
        new = np.arange(seen, want)
        for k, pid in enumerate(new):
            door = (k % 7) if (want - seen) % 7 == 0 else None
            if door is None or p["exited"][pid]:
                continue
            ci, cj = int(np.floor(np.float32(p["x"][pid]) / np.float32(sc.dx))), \
                int(np.floor(np.float32(p["y"][pid]) / np.float32(sc.dx)))
            # visitors entered in this step have not moved yet
            assert cj * sc.nx + ci == sc.door_cells[door], (pid, door)
            assert p["vx"][pid] == 0.0 and p["vy"][pid] == 0.0
            assert 8 <= p["fsm"][pid] < 15 and p["role"][pid] == 0
        seen = want


def test_no_entries_without_trigger_mode_and_capacity_refusals(oracle_mod):
    """evac_trigger = 0 (everyone evacuates from t = 0): nobody enters.  A
    capacity of 5 ids: the rest of the admissions are refused and counted."""
    sc = _empty_centre()
    sc.evac_trigger = 0
    o = oracle_mod.Oracle(sc)
    o.step(30)
    assert o.flow_counts()["n_ids"] == 0
    sc = _empty_centre(capacity=5)
    o = oracle_mod.Oracle(sc)
    o.step(30)
    fc = o.flow_counts()
    assert fc["n_ids"] == 5 and fc["refused"] == 7 * (30 // 6) - 5


def _corridor(length=40, v0=1.2):
    """A 1-cell-high walkable corridor (cells of 1 m), door 0 at its west end,
    door 1 at its east end; no entries (period longer than the run)."""
    nx, ny = length, 3
    sc = S._base("corridor", nx, ny, 1.0, 1e6, 5)
    sc.walkable[:] = 0
    sc.walkable[1, :] = 1
    sc.z[sc.walkable == 0] = 2.0
    sc.door_cells = np.array([1 * nx + 0, 1 * nx + nx - 1], np.int32)
    sc.door_of = np.array([0, 1], np.int32)
    sc.n_doors, sc.entry_period, sc.evac_trigger = 2, 1e5, 1
    sc.ped_noise = 0.0
    p = S.empty_peds(2)
    p["x"][:] = [20.5, 0.5]
    p["y"][:] = 1.5
    p["v0"][:] = v0
    p["fsm"][:] = [9, 8]  # bound for door 1 (east); the second stands in door 0, bound for it
    sc.peds = p
    return sc


def test_lone_visitor_walks_to_its_door_and_leaves(oracle_mod):
    """A visitor 18.5 m from its door at 1.2 m/s in 1 s steps (relaxation
    complete in one step, no noise, no neighbour within 1 m): x grows by 1.2 m
    per step until the last cell, where it slows to reach the door cell's
    centre; it leaves in the step it enters the door cell (step 16: 20.5 +
    15 x 1.2 = 38.5 is the door cell's west edge, so step 16 crosses it).  A
    visitor standing in the door it is bound for leaves at its first step."""
    sc = _corridor()
    o = oracle_mod.Oracle(sc)
    o.step(1)
    p = o.peds()
    assert p["exited"][1] == 2 and o.flow_counts()["n_left"] == 1
    xs = [p["x"][0]]
    for k in range(2, 40):
        o.step(1)
        p = o.peds()
        if p["exited"][0]:
            break
        xs.append(p["x"][0])
    assert p["exited"][0] == 2 and k == 16, (k, xs)
    assert np.allclose(np.diff(xs), 1.2, atol=1e-12)
    assert int(np.floor(p["x"][0])) == 39
    fc = o.flow_counts()
    assert fc["n_left"] == 2 and fc["n_active"] == 0 and fc["n_exited"] == 0


def test_visitors_leave_only_through_their_drawn_door(oracle_mod):
    """600 s of entry/exit flow in the empty centre: ids are conserved at
    every step, visitors leave, and each one gone stands in a cell of the
    door it was bound for."""
    sc = _empty_centre(period=6.0, t_end=600.0)
    o = oracle_mod.Oracle(sc)
    door_of_cell = {int(c): int(d) for c, d in zip(sc.door_cells, sc.door_of)}
    while o.t_ticks < int(600 * TICKS):
        o.step(10)
        fc = o.flow_counts()
        assert fc["n_ids"] == fc["n_active"] + fc["n_left"] + fc["n_exited"]
    p = o.peds()
    gone = np.flatnonzero(p["exited"] == 2)
    assert gone.size > 50 and fc["n_exited"] == 0
    for pid in gone:
        ci = int(np.floor(np.float32(p["x"][pid]) / np.float32(sc.dx)))
        cj = int(np.floor(np.float32(p["y"][pid]) / np.float32(sc.dx)))
        assert door_of_cell.get(cj * sc.nx + ci) == int(p["fsm"][pid]) - 8, pid


def test_first_water_stops_entries_and_turns_visitors_into_evacuees(oracle_mod):
    """A depth hydrograph reaches the breach at 40 s: the step that first sees
    water admits nobody, no visitor enters afterwards, and from that step on
    every evacuee heads for the emergency exit (task 0)."""
    sc = S.shopping_centre(64, 5.0, 0, 0, 3, 400.0, hydro=([0.0, 40.0, 41.0, 400.0], [0.0, 0.0, 1.0, 1.0]))
    S.with_doors(sc, 7, 6.0)
    o = oracle_mod.Oracle(sc)
    entered_at_wet = None
    while o.t_ticks < int(200 * TICKS):
        before = o.flow_counts()["n_entered"]
        wet_before = o.counters()["wet"]
        o.step(1)
        fc = o.flow_counts()
        if o.counters()["wet"]:
            if entered_at_wet is None:
                entered_at_wet = before
                assert not wet_before
            assert fc["n_entered"] == entered_at_wet
            p = o.peds()
            live = (p["exited"] == 0) & (p["role"] == 0)
            assert np.all(p["fsm"][live] == 0)
    assert entered_at_wet is not None and entered_at_wet >= 7 * 6
