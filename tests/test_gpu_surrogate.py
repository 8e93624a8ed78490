"""The learned surrogate's tensor-core (tcgen05) forward and training kernels
against the FP64 oracle of the same conv net."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_1908_05232_b300 as P
    P.build.build()
    oracle.build()
    return torch, P, oracle


def _emulated_forward(O, layers, x):
    """Oracle conv net with the GPU's roundings: BF16 weights and inputs, BF16
    activations between layers, FP32-exact bias; output times 0.1."""
    h = bf16(x).astype(np.float64)
    for l, (w, b) in enumerate(layers):
        h = O.conv3x3(h, bf16(w).astype(np.float64), b.astype(np.float64), relu=l + 1 < len(layers))
        if l + 1 < len(layers):
            h = bf16(h).astype(np.float64)
    return 0.1 * h


@pytest.mark.parametrize("shape", [(2, 40, 150), (1, 11, 11), (1, 20, 301)])
def test_tc_forward_matches_oracle(env, shape):
    torch, P, O = env
    B, H, W = shape
    rng = np.random.default_rng(H * W)
    sur = P.Surrogate(seed=3)
    p = sur.params()
    p[:] = rng.normal(0, 1, p.size).astype(np.float32) * np.float32(0.15)
    sur.set_params(p)
    x = np.stack([rng.uniform(0, 1.2, (B, H, W)), rng.uniform(-1, 1, (B, H, W)),
                  rng.uniform(-1, 1, (B, H, W)), rng.uniform(0, 0.6, (B, H, W))], axis=-1).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros((B, H - 10, W - 10, 3), dtype=torch.float32, device="cuda")
    sur.forward(xd, yd)
    y = yd.cpu().numpy()
    layers = sur.layers(p)
    for b in range(B):
        ref = _emulated_forward(O, layers, x[b])
        err = np.abs(y[b] - ref).max()
        assert err <= 5e-3 * max(1e-3, np.abs(ref).max()), (b, err, np.abs(ref).max())
