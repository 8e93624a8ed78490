"""What the trained net gains over the method without it: trained on the GPU
(the package's own forward/backward/Adam kernels) on plain-solver trajectories
of shopping-centre scenarios, its 8-step depth change on a held-out scenario
is compared with persistence (no change over the window) -- the forecast
available without the net."""
import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_05232_b300 as P
    from paper_1908_05232_b300 import surrogate_train as T
    P.build.build()
    return torch, P, T


def test_trained_net_beats_persistence(env):
    torch, P, T = env
    pairs = []
    for seed, peak in ((2, 0.8), (3, 1.2)):
        sc = S.shopping_centre(256, 0.5, 2000, 0, seed, 1800.0, peak_depth=peak)
        pr, c = T.trajectory_pairs(sc, T.DT_DEFAULT, every=128, n_pairs=48, skip_steps=512)
        assert c["cfl_exceeded"] == 0
        pairs += pr
    sur = P.Surrogate(seed=0)
    losses = T.train(sur, T.CropSampler(pairs, seed=0), steps=1200, batch=32, lr=2e-3, lr_end=2e-5)
    assert np.isfinite(losses).all()
    held, _ = T.trajectory_pairs(S.shopping_centre(256, 0.5, 2000, 0, 7, 1800.0, peak_depth=1.0), T.DT_DEFAULT,
                                 every=128, n_pairs=12, skip_steps=768)
    net_sq, per_sq = 0.0, 0.0
    for x, d in held:
        y = torch.empty((1, x.shape[0] - 10, x.shape[1] - 10, 3), dtype=torch.float32, device="cuda")
        sur.forward(x[None].contiguous(), y)
        net_sq += float(((y[0, ..., 0] - d[..., 0]) ** 2).sum())
        per_sq += float((d[..., 0] ** 2).sum())
    assert per_sq > 0
    # the net's squared depth error over the held-out windows, relative to
    # persistence's (1.0 = no gain)
    ratio = net_sq / per_sq
    print("held-out depth error: net / persistence (squared) = %.3f" % ratio)
    assert ratio < 0.6, ratio
