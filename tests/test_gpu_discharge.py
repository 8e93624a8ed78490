"""The discharge breach (Section 3.1, the paper's inflow form) on the GPU
through the C ABI, against the FP64 oracle: one step and free runs of random
wet states whose edges carry breaches on every side, the exact inflow volume
of a paper hydrograph (36,000 m^3), the maximum-HR history of Fig. 5(b), and
exact mirror symmetry of a west / east breach.

Tolerances as in test_gpu_parity: one step 2e-5 m (+2e-6 relative), free runs
1e-4 m; the domain volume in FP32 cells within 1e-5 relative of the closed
form, the FP64 boundary accumulators within 1e-6."""
import math

import numpy as np
import pytest

import scenarios as S
from tests.conftest import read_golden

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


def _assert_close(sim, o, atol, rtol=0.0):
    for a, name in zip(_fields(sim), ("h", "hu", "hv")):
        b = o.field(name)
        err = np.abs(a.astype(np.float64) - b)
        assert np.all(err <= atol + rtol * np.abs(b)), (name, err.max(), np.unravel_index(err.argmax(), err.shape))


def _breached_state(nx, ny, seed):
    """A rough wet state with a breach on each edge (south and west feed in;
    north and east too), a triangular hydrograph at its rise."""
    sc = S.random_wet_state(nx, ny, dx=0.5, seed=seed, bc=(0, 1, 0, 0))
    S.with_discharge_breach(sc, "south", nx // 5, nx // 3, 12.0, 80.0, h_inflow=0.8)
    sc.bc_w[ny // 4: ny // 4 + ny // 3] = S.BC_DISCHARGE
    sc.bc_n[2: 2 + nx // 6] = S.BC_DISCHARGE
    sc.bc_e[ny // 2: ny // 2 + 5] = S.BC_DISCHARGE
    sc.t0_ticks = 10 << 20
    return sc


@pytest.mark.parametrize("shape", [(150, 70), (67, 131), (5, 3)])
def test_discharge_breach_one_step_and_free_run(P, O, shape):
    nx, ny = shape
    sc = _breached_state(nx, ny, seed=nx + ny)
    o = O.Oracle(sc)
    o.step(1)
    sim = P.from_scenario(sc)
    sim.step(1)
    sim.synchronize()
    assert sim.counters()["t_ticks"] == o.t_ticks
    _assert_close(sim, o, 2e-5, 2e-6)
    # the free run on a fixed step (both sides take the same dt; in CFL mode the
    # FP32 decision may round to a neighbouring tick now and then)
    sc.dt_fixed_ticks = 1 << 15
    o = O.Oracle(sc)
    o.step(200)
    sim = P.from_scenario(sc)
    sim.step(200)
    sim.synchronize()
    c = sim.counters()
    assert c["t_ticks"] == o.t_ticks and c["cfl_exceeded"] == 0
    _assert_close(sim, o, 1e-4)
    m, q = sim.mass()
    assert math.isclose(q, o.boundary_inflow(), rel_tol=1e-5, abs_tol=1e-6)
    assert math.isclose(m, o.mass(), rel_tol=1e-5)


def test_discharge_paper_hydrograph_volume(P, O):
    """The (160 m^3/s, 7.5 min) hydrograph into a walled basin: the water
    held once it has passed is 1/2 Q_peak t_inflow = 36,000 m^3."""
    q_peak, T, _, _, B, vol = [float(v) for v in read_golden("paper_hydrographs.txt")[3]]
    sc = S.breach_basin(n=64, dx=5.0, breach_cells=int(B / 5.0), q_peak=q_peak, t_inflow=T)
    sim = P.from_scenario(sc)
    while sim.counters()["t_ticks"] < int((T + 20.0) * (1 << 20)):
        sim.step(64)
    m, q = sim.mass()
    c = sim.counters()
    assert c["neg_depth"] == 0 and c["error_flags"] == 0
    assert math.isclose(q, vol, rel_tol=1e-6), q
    assert math.isclose(m, vol, rel_tol=1e-5), m
    o = O.Oracle(sc)
    o.step(c["step"])
    assert abs(o.t_ticks - c["t_ticks"]) <= c["step"]  # neighbouring ticks now and then
    _assert_close(sim, o, 1e-4)


def test_max_hr_history(P, O):
    """The maximum-HR time history (Fig. 5(b)) of a breach filling a basin,
    sampled every 20 s, against the oracle's (a fixed 0.25 s step on both
    sides, so the samples fall on the same steps)."""
    sc = S.breach_basin(n=64, dx=5.0, breach_cells=20, q_peak=160.0, t_inflow=450.0)
    sc.dt_fixed_ticks = 1 << 18  # 0.25 s on both sides
    sim = P.from_scenario(sc)
    o = O.Oracle(sc)
    hist_g, hist_o = [], []
    for k in range(1, 13):
        t_k = int(20.0 * k * (1 << 20))
        while sim.counters()["t_ticks"] < t_k:
            sim.step(1)
        while o.t_ticks < t_k:
            o.step(1)
        assert sim.counters()["t_ticks"] == o.t_ticks
        hist_g.append(sim.max_hr())
        hist_o.append(o.max_hr())
    hist_g, hist_o = np.array(hist_g), np.array(hist_o)
    assert hist_o.max() > 0.5
    assert np.allclose(hist_g, hist_o, rtol=1e-4, atol=1e-5), (hist_g, hist_o)


def test_discharge_mirror_symmetry_exact(P):
    """A breach on the west edge and its mirror on the east edge give
    bit-mirrored fields."""
    sc = S.random_wet_state(97, 53, dx=0.5, seed=31, bc=(0, 1, 0, 0))
    S.with_discharge_breach(sc, "west", 10, 20, 9.0, 60.0, h_inflow=0.7)
    m = sc.copy()
    for f in ("z", "h", "hu", "hv", "n0"):
        setattr(m, f, np.ascontiguousarray(getattr(sc, f)[:, ::-1]))
    m.hu = -m.hu
    m.bc_w, m.bc_e = sc.bc_e.copy(), sc.bc_w.copy()
    m.bc_s, m.bc_n = sc.bc_s[::-1].copy(), sc.bc_n[::-1].copy()
    a, b = P.from_scenario(sc), P.from_scenario(m)
    a.step(80)
    b.step(80)
    a.synchronize()
    b.synchronize()
    assert a.counters()["t_ticks"] == b.counters()["t_ticks"]
    ha, hua, hva = _fields(a)
    hb, hub, hvb = _fields(b)
    assert np.array_equal(ha, hb[:, ::-1])
    assert np.array_equal(hua, -hub[:, ::-1])
    assert np.array_equal(hva, hvb[:, ::-1])


def test_discharge_rejected_by_surrogate_and_bad_tables(P):
    from paper_1908_05232_b300 import _native as N
    sc = S.breach_basin(n=32, dx=5.0, breach_cells=8)
    sim = P.from_scenario(sc)
    for t, q, h in (([0.0, 0.0], [1.0, 1.0], 1.0), ([0.0, 1.0], [-1.0, 0.0], 1.0), ([0.0], [1.0], 0.0)):
        with pytest.raises(N.FloodPedError):
            N.fp_set_discharge(sim.h, t, q, h)
    sim.set_fixed_dt(2.0 ** -5)
    sur = P.Surrogate(seed=1)
    with pytest.raises(N.FloodPedError):
        sim.surrogate_advance(sur, 1)
    sur.close()
    sim.close()
