"""Failure detection on the GPU without a GPU fault: a non-finite water state
and a bounded grid-barrier wait that runs out are reported through the C ABI's
status codes (FP_ENAN, FP_ETIMEOUT), reported once, and leave the handle
usable -- after the state is set again, the simulation steps to the same
bytes as a fresh one.

The timeout is made on purpose by lowering the persistent kernel's
grid-barrier poll limit to zero: a CTA that does not find the barrier
complete on its first poll gives up, sets the error bit and leaves the kernel
(no asynchronous copy is in flight at a barrier), and the others follow at
their next barrier.  No trap, no fault, no unbounded wait.
"""
import ctypes

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


def _fields(sim):
    return [sim.field(k) for k in (0, 1, 2)]


def _restore(P, sim, sc):
    """Put a scenario's start state back into a simulation that ran."""
    from paper_1908_05232_b300 import _native as N
    c = np.ascontiguousarray
    N.fp_set_state(sim.h, c(sc.h, np.float32), c(sc.hu, np.float32), c(sc.hv, np.float32))
    N.fp_clear_pedestrians(sim.h)
    if sc.n_peds:
        sim.add_pedestrians(P.ped_records(sc.peds))
    N.fp_set_time(sim.h, sc.t0_ticks, sc.step0)


def _same_run(P, sim, sc, n, mode=None):
    """sim (restored to sc's start) and a fresh simulation of sc give the same bytes after n steps."""
    fresh = P.from_scenario(sc, mode=mode)
    sim.step(n)
    fresh.step(n)
    sim.synchronize()
    fresh.synchronize()
    assert sim.counters()["t_ticks"] == fresh.counters()["t_ticks"]
    for a, b in zip(_fields(sim), _fields(fresh)):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    pa, pb = sim.peds(), fresh.peds()
    assert np.array_equal(pa.view(np.uint8), pb.view(np.uint8))
    fresh.close()


def test_nan_state_reports_enan_once_and_recovers(P):
    from paper_1908_05232_b300 import _native as N
    sc = S.random_wet_state(70, 41, dx=0.5, seed=9)
    sc = S.random_crowd(sc, 40, seed=9)
    sim = P.from_scenario(sc)
    h = sc.h.copy()
    h[17, 23] = np.nan
    h[40, 69] = np.inf
    N.fp_set_state(sim.h, h, np.ascontiguousarray(sc.hu), np.ascontiguousarray(sc.hv))
    sim.step(3)
    assert N.lib().fp_synchronize(sim.h) == N.FP_ENAN
    assert b"non-finite" in N.lib().fp_last_error(sim.h)
    # reported once; the handle takes a valid state and steps on exactly
    assert N.lib().fp_synchronize(sim.h) == N.FP_OK
    _restore(P, sim, sc)
    _same_run(P, sim, sc, 40)
    assert sim.counters()["error_flags"] == 0
    sim.close()


def test_grid_barrier_wait_runs_out_reports_etimeout_and_recovers(P):
    from paper_1908_05232_b300 import _native as N
    sc = S.plain_coupled_128(seed=2, n_peds=300, nx=96, ny=80)
    sim = P.from_scenario(sc, mode=N.FP_MODE_PERSISTENT)
    sim.step(20)
    sim.synchronize()
    with pytest.raises(N.FloodPedError):
        N.fp_set_barrier_wait_limit(sim.h, -1)
    N.fp_set_barrier_wait_limit(sim.h, 0)
    sim.step(6)
    assert N.lib().fp_synchronize(sim.h) == N.FP_ETIMEOUT
    assert b"timed out" in N.lib().fp_last_error(sim.h)
    assert N.lib().fp_synchronize(sim.h) == N.FP_OK
    N.fp_set_barrier_wait_limit(sim.h, 1 << 22)
    _restore(P, sim, sc)
    _same_run(P, sim, sc, 30, mode=N.FP_MODE_PERSISTENT)
    # and the per-step kernels on the same handle after the failed launch
    N.fp_set_step_mode(sim.h, N.FP_MODE_KERNELS)
    _restore(P, sim, sc)
    _same_run(P, sim, sc, 30)
    sim.close()


def test_batch_persistent_barrier_wait_runs_out(P):
    """The batch's persistent kernel with member 0's barrier wait limit at 0
    polls: every wait gives up at once (no spin), fp_batch_synchronize reports
    FP_ETIMEOUT once, and the batch steps again afterwards."""
    from paper_1908_05232_b300 import _native as N
    scs = [S.plain_coupled_128(seed=4, n_peds=100, nx=80 + 16 * k, ny=64) for k in range(2)]
    sims = [P.from_scenario(sc) for sc in scs]
    b = P.Batch(sims, mode=N.FP_MODE_PERSISTENT)
    b.step(8)
    b.synchronize()
    N.fp_set_barrier_wait_limit(sims[0].h, 0)
    b.step(4)
    assert N.lib().fp_batch_synchronize(b.h) == N.FP_ETIMEOUT
    assert N.lib().fp_batch_synchronize(b.h) == N.FP_OK
    N.fp_set_barrier_wait_limit(sims[0].h, 1 << 22)
    b.set_mode(N.FP_MODE_KERNELS)
    b.step(8)
    b.synchronize()
    b.set_mode(N.FP_MODE_PERSISTENT)
    b.step(8)
    b.synchronize()
    b.close()
    for s in sims:
        s.close()


def test_batch_reports_member_error(P):
    """A member's non-finite state surfaces from the batch's synchronisation."""
    from paper_1908_05232_b300 import _native as N
    scs = [S.random_wet_state(40 + 8 * k, 30, dx=0.5, seed=20 + k) for k in range(3)]
    sims = [P.from_scenario(sc) for sc in scs]
    h = scs[1].h.copy()
    h[5, 5] = np.nan
    N.fp_set_state(sims[1].h, h, np.ascontiguousarray(scs[1].hu), np.ascontiguousarray(scs[1].hv))
    b = P.Batch(sims)
    b.step(4)
    rc = N.lib().fp_batch_synchronize(b.h)
    assert rc == N.FP_ENAN
    b.close()
    for s in sims:
        s.close()
