"""Pins of the oracle's second-order scheme (the cited scheme at full order:
MUSCL reconstruction, hydrostatic reconstruction with the centred bed-slope
term, two-stage Runge-Kutta), a build-added option beside the paper's first
order.  CPU only.

What fixes the values: a lake at rest over an uneven bed with emerged dry
bumps stays exactly at rest (the well-balanced property); mass is conserved
to round-off in a closed box and balances the boundary volumes otherwise;
mirror symmetry is exact; on a smooth wave the error falls at second order
under refinement (the first-order scheme at first order: a dropped slope or a
one-stage time step fails); the Stoker dam break is closer to its closed form
than the first-order scheme on the same grid."""
import math

import numpy as np
import pytest

import scenarios as S
from tests.test_oracle_pins import _stoker


def _order2(sc):
    sc.order = 2
    return sc


def test_lake_at_rest_exact(oracle_mod):
    sc = _order2(S.closed_basin(40, 31, dx=1.0, seed=3))
    assert (sc.z > 0.75).any(), "needs emerged dry bumps"
    o = oracle_mod.Oracle(sc)
    eta0 = o.h + o.z
    wet = o.h > 0
    o.step(150)
    assert np.all(o.hu == 0.0) and np.all(o.hv == 0.0)
    assert np.array_equal((o.h + o.z)[wet], eta0[wet])
    assert np.all(o.h[~wet] == 0.0)


def test_mass_closed_and_open(oracle_mod):
    sc = _order2(S.random_wet_state(37, 29, dx=0.5, seed=11, bc=(0, 0, 0, 0)))
    o = oracle_mod.Oracle(sc)
    m0 = o.mass()
    o.step(300)
    assert o.counters()["neg_depth"] == 0
    assert abs(o.mass() - m0) <= 1e-12 * m0
    sc = _order2(S.random_wet_state(33, 27, dx=1.0, seed=5))
    o = oracle_mod.Oracle(sc)
    m0 = o.mass()
    o.step(300)
    assert abs(o.mass() - (m0 + o.boundary_inflow())) <= 1e-11 * m0


@pytest.mark.parametrize("axis", ["x", "y"])
def test_mirror_symmetry_exact(oracle_mod, axis):
    sc = _order2(S.random_wet_state(23, 19, dx=0.7, seed=21, bc=(2, 1, 0, 1)))
    m = sc.copy()
    if axis == "x":
        for f in ("z", "h", "hu", "hv", "n0"):
            setattr(m, f, getattr(sc, f)[:, ::-1].copy())
        m.hu = -m.hu
        m.bc_w, m.bc_e = sc.bc_e.copy(), sc.bc_w.copy()
        m.bc_s, m.bc_n = sc.bc_s[::-1].copy(), sc.bc_n[::-1].copy()
    else:
        for f in ("z", "h", "hu", "hv", "n0"):
            setattr(m, f, getattr(sc, f)[::-1, :].copy())
        m.hv = -m.hv
        m.bc_s, m.bc_n = sc.bc_n.copy(), sc.bc_s.copy()
        m.bc_w, m.bc_e = sc.bc_w[::-1].copy(), sc.bc_e[::-1].copy()
    a, b = oracle_mod.Oracle(sc), oracle_mod.Oracle(m)
    a.step(40)
    b.step(40)
    fl = (lambda f: f[:, ::-1]) if axis == "x" else (lambda f: f[::-1, :])
    sgn_u, sgn_v = (-1, 1) if axis == "x" else (1, -1)
    assert np.array_equal(a.field("h"), fl(b.field("h")))
    assert np.array_equal(a.field("hu"), sgn_u * fl(b.field("hu")))
    assert np.array_equal(a.field("hv"), sgn_v * fl(b.field("hv")))


def _smooth_wave(oracle_mod, nx, order, L=20.0, T=1.0):
    """A smooth hump of water (0.1 m on 1 m, width 2 m) on a flat frictionless
    bed, walls far away; fixed step proportional to dx (Courant number 0.27)
    to T = 1 s, before the wave steepens into a bore.  Returns h along x."""
    dx = L / nx
    sc = S.dam_break_1d(nx=nx, ny=1, dx=dx, h_left=1.0, h_right=1.0, t_end=T)
    x = (np.arange(nx) + 0.5) * dx
    sc.h[:] = (1.0 + 0.1 * np.exp(-((x - 0.5 * L) / 2.0) ** 2)).astype(np.float32)[None, :]
    sc.n0[:] = 0.0
    sc.order = order
    sc.dt_fixed_ticks = int(round((1 << 20) * 0.015625 * 100.0 / nx))  # 2^-6 s at 100 cells, halving with dx
    o = oracle_mod.Oracle(sc)
    o.step(100000)
    assert abs(o.t - T) < 1e-12
    return o.field("h")[0]


@pytest.mark.parametrize("order,lo,hi", [(2, 1.7, 2.3), (1, 0.8, 1.2)])
def test_smooth_wave_convergence_order(oracle_mod, order, lo, hi):
    """Errors against a 3200-cell solution (block means): the observed order
    of the second-order scheme near 2, of the first-order scheme near 1."""
    ref = _smooth_wave(oracle_mod, 3200, order)
    errs = []
    for nx in (100, 200, 400):
        h = _smooth_wave(oracle_mod, nx, order)
        r = ref.reshape(nx, -1).mean(axis=1)
        errs.append(np.abs(h - r).sum() * (20.0 / nx))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(lo < q < hi for q in rates), (errs, rates)


def test_stoker_closer_than_first_order(oracle_mod):
    g = float(np.float32(9.81))
    errs = {}
    for order in (1, 2):
        nx, L, T = 400, 100.0, 4.0
        dx = L / nx
        sc = S.dam_break_1d(nx=nx, ny=3, dx=dx, h_left=1.0, h_right=0.1, t_end=T)
        sc.order = order
        o = oracle_mod.Oracle(sc)
        o.step(100000)
        xc = (np.arange(nx) + 0.5) * dx - 0.5 * L
        h = o.field("h")
        assert np.array_equal(h[0], h[1]) and np.array_equal(h[0], h[2])
        errs[order] = np.abs(h[1] - _stoker(xc, T, 1.0, 0.1, g)).sum() * dx
    assert errs[2] < 0.7 * errs[1], errs
