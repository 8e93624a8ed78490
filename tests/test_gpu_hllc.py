"""The HLLC interface flux (fp_config.riemann = FP_RIEMANN_HLLC) on the GPU
through the C ABI, against the FP64 oracle's HLLC: one step and a fixed-step
free run of random wet states with every boundary type, the shear wave it
advects upwind, exact lake at rest and mirror symmetry, and the same bytes in
every step mode.  Tolerances as in test_gpu_parity."""
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
        assert np.all(err <= atol + rtol * np.abs(b)), (name, err.max())


@pytest.mark.parametrize("shape", [(150, 70), (67, 131), (5, 3)])
def test_hllc_one_step_and_free_run(P, O, shape):
    nx, ny = shape
    sc = S.random_wet_state(nx, ny, dx=0.5, seed=nx * ny, bc=(2, 1, 0, 1))
    sc.riemann = 1
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
    assert sim.counters()["t_ticks"] == o.t_ticks
    _close(sim, o, 1e-4)


def test_hllc_shear_wave_upwind(P):
    """Uniform depth and normal velocity, the tangential velocity jumping from
    +1 to -1: one HLLC step is first-order upwind advection of hv at the flow
    speed; HLL smears the jump."""
    nx = 64
    sc = S.closed_basin(nx, 3, dx=1.0, wet=False, bumps=False)
    sc.h[:] = 1.0
    sc.hu[:] = 0.5
    sc.hv[:, : nx // 2] = 1.0
    sc.hv[:, nx // 2:] = -1.0
    sc.n0[:] = 0.0
    sc.bc_s[:], sc.bc_n[:], sc.bc_w[:], sc.bc_e[:] = 1, 1, 1, 1
    sc.riemann = 1
    sim = P.from_scenario(sc)
    sim.step(1)
    sim.synchronize()
    lam = sim.counters()["t_ticks"] / float(1 << 20) / sc.dx
    v0 = np.where(np.arange(nx) < nx // 2, 1.0, -1.0)
    want = v0 - lam * 0.5 * (v0 - np.concatenate([[v0[0]], v0[:-1]]))
    hv = sim.field(2)
    assert np.abs(hv - want[None, :]).max() <= 1e-6
    sc.riemann = 0
    b = P.from_scenario(sc)
    b.step(1)
    b.synchronize()
    assert np.abs(b.field(2)[1] - want).max() > 1e-2


def test_hllc_lake_at_rest_and_mirror(P):
    sc = S.closed_basin(150, 70, dx=1.0, seed=3)
    sc.riemann = 1
    sim = P.from_scenario(sc)
    sim.step(200)
    h, hu, hv = _fields(sim)
    z = sim.field(3)
    wet = sc.h > 0
    assert np.all(hu == 0) and np.all(hv == 0)
    assert np.array_equal((h + z)[wet], (sc.h + sc.z)[wet])
    sc = S.random_wet_state(133, 77, dx=0.7, seed=21, bc=(2, 1, 0, 1))
    sc.riemann = 1
    m = sc.copy()
    for f in ("z", "h", "hu", "hv", "n0"):
        setattr(m, f, np.ascontiguousarray(getattr(sc, f)[:, ::-1]))
    m.hu = -m.hu
    m.bc_w, m.bc_e = sc.bc_e.copy(), sc.bc_w.copy()
    m.bc_s, m.bc_n = sc.bc_s[::-1].copy(), sc.bc_n[::-1].copy()
    a, b = P.from_scenario(sc), P.from_scenario(m)
    a.step(60)
    b.step(60)
    a.synchronize()
    b.synchronize()
    ha, hua, hva = _fields(a)
    hb, hub, hvb = _fields(b)
    assert np.array_equal(ha, hb[:, ::-1]) and np.array_equal(hua, -hub[:, ::-1]) and np.array_equal(hva, hvb[:, ::-1])


def test_hllc_same_bytes_in_every_mode(P):
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=5)
    sc.riemann = 1
    a = P.from_scenario(sc, mode=N.FP_MODE_KERNELS)
    b = P.from_scenario(sc, mode=N.FP_MODE_PERSISTENT)
    c = P.from_scenario(sc)
    a.step(150)
    b.step(150)
    batch = P.Batch([c])
    batch.step(150)
    batch.synchronize()
    for x, y, w in zip(_fields(a), _fields(b), _fields(c)):
        assert np.array_equal(x, y) and np.array_equal(x, w)
    assert np.array_equal(a.peds(), b.peds()) and np.array_equal(a.peds(), c.peds())
    batch.close()
