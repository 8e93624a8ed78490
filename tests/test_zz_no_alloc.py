"""The allocation-free water-volume entry point (fp_water_volume_noalloc),
called through the C ABI, against the library's regular volume read
(fp_read_state FP_FIELD_MASS) of the same depth grid.

It is meant for callers that may not allocate device memory through this
library (their device memory belongs to a host framework's pool, or is sized
once at start-up).  Both results are FP64 sums of the same FP32 depths in a
different order, so they agree to ~1e-15 relative; the check uses 1e-12,
tighter than the 2e-6 relative the other volume tests allow.  This file is
collected last so that a run stopping at its first failure has already run
every other test."""
import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_05232_b300 as P
    P.build.build()
    return torch, P


def test_noalloc_volume_matches_regular_read_twice():
    torch, P = _setup()
    from paper_1908_05232_b300 import _native as N
    sc = S.random_wet_state(300, 170, dx=0.5, seed=31)
    sim = P.from_scenario(sc)
    sim.step(20)
    sim.synchronize()
    ref, _ = sim.mass()
    depth = torch.empty((sc.ny, sc.nx), dtype=torch.float32, device="cuda")
    N.fp_read_state(sim.h, N.FP_FIELD_H, depth)
    torch.cuda.synchronize()
    for _ in range(2):  # the second call reuses the scratch the first one left behind
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        N.fp_water_volume_noalloc(depth, sc.nx, sc.ny, sc.nx, sc.dx, out)
        torch.cuda.synchronize()
        assert abs(out.item() - ref) <= 1e-12 * ref, (out.item(), ref)
    # a padded row pitch gives the same volume
    padded = torch.zeros((sc.ny, sc.nx + 13), dtype=torch.float32, device="cuda")
    padded[:, :sc.nx] = depth
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    N.fp_water_volume_noalloc(padded, sc.nx, sc.ny, sc.nx + 13, sc.dx, out)
    torch.cuda.synchronize()
    assert abs(out.item() - ref) <= 1e-12 * ref


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, P = _setup()
    from paper_1908_05232_b300 import _native as N
    depth = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(N.FloodPedError, match="FP_NOALLOC_MAX_ROWS"):
        N.fp_water_volume_noalloc(depth, 4, 65537, 4, 0.5, out)
    with pytest.raises(N.FloodPedError):
        N.fp_water_volume_noalloc(depth, 4, 4, 3, 0.5, out)
