"""Free-running coupled parity against the FP64 oracle, step by step.

The plain coupled workload of 128 x 128 cells with 256 evacuees (and a
low-density variant with 32) runs 1000 coupled steps on the GPU and in the
oracle in lock step; after every step every pedestrian's integers (hazard
state, exit) must be identical and its position within 1e-3 m, and the flood
fields within 1e-4 m at the checkpoints.  The CFL step is an FP32 decision on
states that differ by FP32 against FP64 rounding, so the clocks may come to
differ by a tick (1e-6 s) now and then: up to 100 ticks (1e-4 s) over the
1000 steps are allowed (19 seen).

Where crowd contact makes trajectories diverge (individual paths in a dense
crowd are chaotic under FP32 against FP64 rounding), the test reports the
first divergent step and the pedestrians involved and then checks only the
invariants of the crowd: the dense variant on a fixed 1/8 s step is that case."""
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


def _diverged(g, r, pos_tol):
    dpos = np.maximum(np.abs(g["x"] - r["x"]), np.abs(g["y"] - r["y"]))
    bad = (g["exited"] != r["exited"]) | (g["hr"] != r["hr"]) | (dpos > pos_tol)
    return bad, dpos


def _lockstep(P, O, sc, n, pos_tol=1e-3):
    """Steps both sides n times; returns (first divergence or None, largest
    position difference before it, largest clock difference in ticks)."""
    o = O.Oracle(sc)
    sim = P.from_scenario(sc)
    worst, ticks = 0.0, 0
    for s in range(1, n + 1):
        o.step(1)
        sim.step(1)
        c = sim.counters()
        ticks = max(ticks, abs(c["t_ticks"] - o.t_ticks))
        g, r = sim.peds(), o.peds()
        bad, dpos = _diverged(g, r, pos_tol)
        if bad.any():
            ids = np.nonzero(bad)[0]
            return dict(step=s, ids=ids.tolist(), dpos=dpos[ids].tolist()), worst, ticks, sim, o
        live = r["exited"] == 0
        if live.any():
            worst = max(worst, float(dpos[live].max()))
        if s % 250 == 0:
            for k, name in ((0, "h"), (1, "hu"), (2, "hv")):
                err = np.abs(sim.field(k).astype(np.float64) - o.field(name)).max()
                assert err <= 1e-4, (s, name, err)
    return None, worst, ticks, sim, o


@pytest.mark.parametrize("n_peds", [256, 32])
def test_coupled_1000_steps_lockstep(P, O, n_peds):
    sc = S.plain_coupled_128(seed=1, n_peds=n_peds)
    first, worst, ticks, sim, o = _lockstep(P, O, sc, 1000)
    assert first is None, "first divergence: %s" % first
    assert worst <= 1e-3 and ticks <= 100, (worst, ticks)
    c, oc = sim.counters(), o.counters()
    assert c["n_exited"] == oc["n_exited"] and c["hist"] == oc["hist"]
    assert c["n_exited"] > 0.5 * n_peds  # the run reached the evacuation


def test_dense_fixed_step_divergence_report(P, O):
    """The dense crowd on a fixed 1/8 s step: identical until the first
    divergence, which involves few pedestrians (a contact, not a systematic
    difference); afterwards the crowd keeps its invariants on both sides."""
    sc = S.plain_coupled_128(seed=1)
    sc.dt_fixed_ticks = 1 << 17
    first, worst, ticks, sim, o = _lockstep(P, O, sc, 1000)
    assert ticks == 0 and worst <= 1e-3
    if first is None:
        return
    print("first divergence at step %d, pedestrians %s, position differences %s"
          % (first["step"], first["ids"], ["%.3g" % d for d in first["dpos"]]))
    assert len(first["ids"]) <= 3, first
    # invariants after the divergence, on the GPU side
    left = 1000 - first["step"]
    sim.step(left)
    o.step(left)
    c = sim.counters()
    g = sim.peds()
    assert c["n_active"] + c["n_exited"] == sc.n_peds and c["error_flags"] == 0
    live = g["exited"] == 0
    ii = np.floor(g["x"][live] / np.float32(sc.dx)).astype(int)
    jj = np.floor(g["y"][live] / np.float32(sc.dx)).astype(int)
    assert np.all(sc.walkable[jj, ii] == 1)
    assert abs(c["n_exited"] - o.counters()["n_exited"]) <= 3
