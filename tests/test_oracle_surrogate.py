"""Pins of the oracle's FP64 conv net (the learned surrogate, build-added):
exact special cases of a convolution and central finite differences of the
loss gradient."""
import math

import numpy as np
import pytest


def _net(rng, ch=(4, 6, 5, 3)):
    ws = [rng.normal(0, 0.4, (3, 3, ch[l], ch[l + 1])) for l in range(len(ch) - 1)]
    bs = [rng.normal(0, 0.1, ch[l + 1]) for l in range(len(ch) - 1)]
    return ws, bs


def test_conv_delta_kernel_is_center_crop(oracle_mod):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(9, 7, 3))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[1, 1, c, c] = 1.0
    y = oracle_mod.conv3x3(x, w, np.zeros(3))
    assert np.array_equal(y, x[1:-1, 1:-1, :])


def test_conv_shift_and_sum_of_taps(oracle_mod):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(8, 10, 2))
    w = np.zeros((3, 3, 2, 1))
    w[0, 2, 1, 0] = 1.0          # picks x[i, j+2, 1]
    w[2, 0, 0, 0] = -2.0         # and -2 x[i+2, j, 0]
    y = oracle_mod.conv3x3(x, w, np.array([0.5]))
    want = x[:-2, 2:, 1] - 2.0 * x[2:, :-2, 0] + 0.5
    assert np.allclose(y[..., 0], want, rtol=0, atol=1e-15)


def test_relu_clamps(oracle_mod):
    x = -np.ones((3, 3, 1))
    w = np.ones((3, 3, 1, 1))
    assert oracle_mod.conv3x3(x, w, np.zeros(1), relu=True)[0, 0, 0] == 0.0
    assert oracle_mod.conv3x3(x, w, np.zeros(1), relu=False)[0, 0, 0] == -9.0


def test_loss_gradient_finite_differences(oracle_mod):
    rng = np.random.default_rng(2)
    ws, bs = _net(rng)
    x = rng.normal(size=(12, 11, 4))
    target = rng.normal(size=(6, 5, 3))
    loss, dws, dbs = oracle_mod.net_loss_grad(x, ws, bs, target)
    out = oracle_mod.net_forward(x, ws, bs)
    assert np.isclose(loss, np.mean((out - target) ** 2), rtol=1e-12)
    eps = 1e-6
    for l in range(len(ws)):
        for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (2, 1, ws[l].shape[2] - 1, ws[l].shape[3] - 1)]:
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[l][idx] += eps
            wm[l][idx] -= eps
            lp = oracle_mod.net_loss_grad(x, wp, bs, target)[0]
            lm = oracle_mod.net_loss_grad(x, wm, bs, target)[0]
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - dws[l][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, dws[l][idx])
        k = bs[l].shape[0] - 1
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][k] += eps
        bm[l][k] -= eps
        fd = (oracle_mod.net_loss_grad(x, ws, bp, target)[0] - oracle_mod.net_loss_grad(x, ws, bm, target)[0]) / (2 * eps)
        assert abs(fd - dbs[l][k]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_activation_option_special_cases(oracle_mod):
    """The option that stores hidden activations in BF16: integer activations
    below 256 are BF16 numbers and pass unchanged; 1 + 2^-9 lies halfway
    between the BF16 neighbours 1 and 1 + 2^-7 and rounds to the even one (1);
    1 + 3 * 2^-9 rounds up to 1 + 2^-8 * 2 = 1 + 2^-7."""
    delta = np.zeros((3, 3, 1, 1))
    delta[1, 1, 0, 0] = 1.0
    ws, bs = [delta, delta], [np.zeros(1), np.zeros(1)]
    for v, want in ((37.0, 37.0), (1.0 + 2.0 ** -9, 1.0), (1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7),
                    (-5.0, 0.0)):
        x = np.full((5, 5, 1), v)
        t = np.zeros((1, 1, 1))
        loss_b = oracle_mod.net_loss_grad(x, ws, bs, t, act_bf16=True)[0]
        loss_p = oracle_mod.net_loss_grad(x, ws, bs, t, act_bf16=False)[0]
        assert loss_b == want ** 2, (v, loss_b)
        assert loss_p == max(v, 0.0) ** 2
    rng = np.random.default_rng(3)
    ws2 = [rng.integers(-1, 2, (3, 3, 2, 3)).astype(float), rng.integers(-1, 2, (3, 3, 3, 2)).astype(float)]
    bs2 = [np.zeros(3), np.zeros(2)]
    x = rng.integers(0, 3, (9, 8, 2)).astype(float)
    t = rng.normal(size=(5, 4, 2))
    a = oracle_mod.net_loss_grad(x, ws2, bs2, t, act_bf16=True)
    b = oracle_mod.net_loss_grad(x, ws2, bs2, t, act_bf16=False)
    assert a[0] == b[0]
    for ga, gb in zip(a[1] + a[2], b[1] + b[2]):
        assert np.array_equal(ga, gb)


# --------------------------------------------------------------------------
# The surrogate guard's per-tile mass residual (build-added): closed-form cases
# --------------------------------------------------------------------------
def _channel(oracle_mod, u):
    """A 10 x 3 walled channel of 1 m cells, still bed, water 1 m deep moving at u."""
    import scenarios as S
    sc = S.closed_basin(10, 3, dx=1.0, wet=False, bumps=False)
    sc.h[:] = 1.0
    sc.hu[:] = u
    return sc, oracle_mod.Oracle(sc)


def test_guard_residual_closed_box_redistribution(oracle_mod):
    """Water moved inside a walled box: no volume change, no flow through walls."""
    sc, o = _channel(oracle_mod, 0.0)
    h0 = sc.h.astype(np.float64)
    h1 = h0.copy()
    h1[1, 2] += 0.25
    h1[1, 7] -= 0.25
    z = np.zeros_like(h0)
    r = o.guard_residual((h0, z, z), (h1, z, z), 0, 10, 0, 3, 0, 1 << 18)
    assert r == 0.0


def test_guard_residual_inflow_sign_and_window(oracle_mod):
    """Tile = the channel's east half against the east wall, water flowing in
    from the west half at q = 0.5 m^2/s: the west face carries exactly q (the
    states either side are identical), the wall nothing (a reflected state).
    Unchanged water: residual = window x 3 rows x q / start volume; water raised
    by that inflow: residual 0."""
    sc, o = _channel(oracle_mod, 0.5)
    h0 = sc.h.astype(np.float64)
    hu0 = sc.hu.astype(np.float64)
    z = np.zeros_like(h0)
    t1 = 1 << 18  # 0.25 s
    r = o.guard_residual((h0, hu0, z), (h0, hu0, z), 5, 10, 0, 3, 0, t1)
    assert math.isclose(r, 0.25 * 3 * 0.5 / 15.0, rel_tol=1e-12), r
    h1 = h0.copy()
    h1[:, 5:] += 0.25 * 3 * 0.5 / 15.0
    hu1 = hu0.copy()
    hu1[:, 5:] = 0.5 * h1[:, 5:]  # the same velocity: the west face still carries h u of identical states
    hu1[:, :5] = 0.5
    h1[:, :5] = 1.0
    r = o.guard_residual((h0, hu0, z), (h1, hu1, z), 5, 10, 0, 3, 0, t1)
    # end state's west face: (1, 0.5) | (1.025, 0.5): the HLL average, not exactly q;
    # the residual is then the difference of the two fluxes' mean from q
    assert r < 5e-3, r


def test_guard_residual_floor_of_one_centimetre(oracle_mod):
    """A nearly dry tile: the denominator is 1 cm over the tile's area."""
    sc, o = _channel(oracle_mod, 0.0)
    h0 = np.zeros((3, 10))
    h1 = h0.copy()
    h1[1, 6] = 0.003
    z = np.zeros_like(h0)
    r = o.guard_residual((h0, z, z), (h1, z, z), 5, 10, 0, 3, 0, 1 << 18)
    assert math.isclose(r, 0.003 / (0.01 * 15.0), rel_tol=1e-12), r
