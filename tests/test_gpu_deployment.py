"""Scenario 2 of the paper (Section 3.3) as a batched ensemble on the GPU:
responder groups and barrier thicknesses stepped together until every barrier
is built, then the discharge flood of Section 3.1.  Checked: a reduced study
(2 group sizes x 2 thicknesses on a 48 x 48 shopping centre of 2.59 m cells)
builds every barrier, its deployment times order as they must (more responders
sooner, more layers later, never faster than 60 s per bag and responder), and
one run of it matches the FP64 oracle: in lock step until crowd contact splits
a responder's path, then on the outcome (the same barrier within 5 % of the
deployment time) and on the flood that follows (within 1e-4 m)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_05232_b300 as pkg
    pkg.build.build()
    return pkg


SMALL = dict(fractions=(0.1, 0.3), layers=(1, 2), n=48, dx=2.59, n_peds=100, n_barrier=8, seed=5)


def test_reduced_deployment_study(P):
    from paper_1908_05232_b300 import studies
    res = studies.deployment_study(P, flood_minutes=4.0, **SMALL)
    rows = {(r["responders"], r["layers"]): r for r in res["rows"]}
    assert len(rows) == 4
    for (R, L), r in rows.items():
        assert r["deploy_s"] is not None and r["within_window"], r
        assert r["deploy_s"] >= 60.0 * math.ceil(r["bags"] / R), r
    for L in (1, 2):
        assert rows[(30, L)]["deploy_s"] < rows[(10, L)]["deploy_s"]
    for R in (10, 30):
        assert rows[(R, 2)]["deploy_s"] > rows[(R, 1)]["deploy_s"]
    assert all(r["downstream_depth_m"] >= 0.0 for r in rows.values())


def test_deployment_run_matches_oracle(P):
    """One run of the study (30 responders, 2 layers) against the oracle in
    lock step: identical clocks, bag counts, built layers and responder tasks
    until crowd contact makes a responder reach the depot or the barrier a step
    apart on the two sides (responders walk through a standing crowd on 1 s
    dry steps: individual paths are chaotic under FP32 against FP64 rounding);
    the first such step is reported.  Both sides then build the same barrier
    (the bed identical) within 5 % of each other's deployment time, and the
    flood that follows, started on both sides from the oracle's state at the
    end of the deployment, agrees within 1e-4 m."""
    import oracle
    from paper_1908_05232_b300 import _native as N
    from paper_1908_05232_b300 import studies
    oracle.build()
    (sc, meta), = studies.deployment_scenarios(fractions=(0.3,), layers=(2,), n=48, dx=2.59, n_peds=100,
                                               n_barrier=8, seed=5)
    sim = P.from_scenario(sc)
    o = oracle.Oracle(sc)
    target = len(sc.barrier_cells) * sc.n_layers
    first, t_gpu, t_orc, steps = None, None, None, 0
    while (t_gpu is None or t_orc is None) and steps < 40000:
        sim.step(16)
        o.step(16)
        steps += 16
        c, oc = sim.counters(), o.counters()
        assert c["t_ticks"] == oc["t_ticks"]  # dry 1 s steps on both sides
        if first is None and (c["total_bags"] != oc["total_bags"] or c["applied_layers"] != oc["applied_layers"]
                              or not np.array_equal(sim.peds()["task"], o.peds()["fsm"])):
            first = steps
        if t_gpu is None and c["applied_layers"] >= target:
            t_gpu = c["t_ticks"] / N.TICKS
        if t_orc is None and oc["applied_layers"] >= target:
            t_orc = oc["t_ticks"] / N.TICKS
    print("deployment: first divergence at step", first, "; built after", t_gpu, "s (GPU),", t_orc, "s (oracle)")
    assert first is None or first >= 64
    assert t_gpu is not None and t_orc is not None
    assert abs(t_gpu - t_orc) <= 0.05 * t_orc
    # the same barrier: FP32 against FP64 sums of the noisy bed and the layers
    zg, zo = sim.field(N.FP_FIELD_Z).astype(np.float64), o.field("z")
    assert np.abs(zg - zo).max() <= 1e-6
    raised = (zo - sc.z.astype(np.float64)).reshape(-1)[sc.barrier_cells]
    assert np.allclose(raised, 0.25 * sc.n_layers, atol=1e-6)
    # the discharge flood through the breach from the oracle's end state, a fixed step on both sides
    t0 = o.t
    b0, bw = sc.breach
    sc2 = o.to_scenario()
    sc2.bc_s = np.asarray(sc.bc_s, np.uint8).copy()
    sc2.bc_s[b0:b0 + bw] = N.FP_BC_DISCHARGE
    sc2.q_t = np.array([t0, t0 + 225.0, t0 + 450.0])
    sc2.q_Q = np.array([0.0, 160.0, 0.0])
    sc2.dt_fixed_ticks = 1 << 18
    a, b = P.from_scenario(sc2), oracle.Oracle(sc2)
    a.step(480)
    b.step(480)
    assert a.counters()["t_ticks"] == b.t_ticks
    for k, name in ((0, "h"), (1, "hu"), (2, "hv")):
        err = np.abs(a.field(k).astype(np.float64) - b.field(name)).max()
        assert err <= 1e-4, (name, err)
    assert a.max_hr() > 0.0


def test_hr_history_sampling(P):
    """The maximum-HR time history of a breach filling a basin (Fig. 5(b)'s
    measure): one sample every 6 s of simulated time, zero before the water
    arrives and positive after."""
    import scenarios as S
    from paper_1908_05232_b300 import studies
    sc = S.breach_basin(n=48, dx=5.0, breach_cells=16, q_peak=160.0, t_inflow=450.0)
    hist = studies.hr_history(P, sc, minutes=2.0, every_s=6.0)
    t = np.array([a for a, _ in hist])
    v = np.array([b for _, b in hist])
    assert len(hist) == 20
    assert np.all(np.diff(t) > 0) and np.all(t >= 6.0 * np.arange(1, 21))
    assert v[-1] > 0.0 and np.all(np.isfinite(v))
