"""The learned surrogate's tensor-core (tcgen05) forward and training kernels
against the FP64 oracle of the same conv net."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OUT_SCALE = 2.0 ** -10  # FP_SUR_OUT_SCALE


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


def split(x):
    """The net's input channels: each input rounded to BF16, then the BF16-rounded
    remainders (FP32 subtraction, as the input packing does)."""
    hi = bf16(x)
    lo = bf16(np.asarray(x, np.float32) - hi)
    return np.concatenate([hi, lo], axis=-1)


def _emulated_forward(O, layers, x):
    """Oracle conv net with the GPU's roundings: BF16 weights and split inputs,
    BF16 activations between layers, FP32-exact bias; output times 2^-10."""
    h = split(x).astype(np.float64)
    for l, (w, b) in enumerate(layers):
        h = O.conv3x3(h, bf16(w).astype(np.float64), b.astype(np.float64), relu=l + 1 < len(layers))
        if l + 1 < len(layers):
            h = bf16(h).astype(np.float64)
    return OUT_SCALE * h


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


def _inputs(rng, B, H, W):
    return np.stack([rng.uniform(0, 1.2, (B, H, W)), rng.uniform(-1, 1, (B, H, W)),
                     rng.uniform(-1, 1, (B, H, W)), rng.uniform(0, 0.6, (B, H, W))], axis=-1).astype(np.float32)


@pytest.mark.parametrize("shape,ctas", [((1, 14, 19), 0), ((2, 24, 150), 0), ((2, 24, 150), 4)])
def test_gradients_match_oracle(env, shape, ctas):
    """Loss and every parameter gradient of the CUDA backward against the FP64
    oracle backward, the oracle given the BF16-rounded weights and split inputs
    the tensor cores see, the last layer scaled by the output factor 2^-10, and
    its hidden activations stored in BF16 as on the GPU (the same rounding).
    What remains is FP32 against FP64 accumulation, and hidden values whose
    FP32 and FP64 pre-activations round to different BF16 numbers (or fall on
    either side of zero): 2e-3 relative on these inputs.  With ctas = 4 each
    kernel runs on four CTAs: the weight-gradient kernel then takes 9 work
    items per CTA (36 items of 4 rows x 64 pixels in layer 0), reusing both of
    its staging buffers, and the data-gradient convolution several strips."""
    torch, P, O = env
    B, H, W = shape
    rng = np.random.default_rng(B * H * W)
    sur = P.Surrogate(seed=11)
    sur.set_max_ctas(ctas)
    p = sur.params()
    p[:] = rng.normal(0, 1, p.size).astype(np.float32) * np.float32(0.12)
    sur.set_params(p)
    x = _inputs(rng, B, H, W)
    t = rng.normal(0, 0.05, (B, H - 10, W - 10, 3)).astype(np.float32)
    loss, g = sur.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    layers = sur.layers(p)
    ws = [bf16(w).astype(np.float64) for w, _ in layers]
    bs = [b.astype(np.float64) for _, b in layers]
    ws[-1] = ws[-1] * OUT_SCALE
    bs[-1] = bs[-1] * OUT_SCALE
    ref_loss = 0.0
    ref_g = [np.zeros_like(w) for w in ws] + [np.zeros_like(b) for b in bs]
    for b in range(B):
        lb, dws, dbs = O.net_loss_grad(split(x[b]).astype(np.float64), ws, bs, t[b].astype(np.float64),
                                       act_bf16=True)
        ref_loss += lb / B
        for l in range(len(ws)):
            scale = OUT_SCALE if l == len(ws) - 1 else 1.0
            ref_g[l] += scale * dws[l] / B
            ref_g[len(ws) + l] += scale * dbs[l] / B
    assert abs(loss - ref_loss) <= 1e-4 * ref_loss, (loss, ref_loss)
    tol = 2e-3
    gl = sur.layers(g)
    for l, (dw, db) in enumerate(gl):
        for got, ref in ((dw, ref_g[l]), (db, ref_g[len(ws) + l])):
            rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
            assert rel <= tol, (l, rel)
            # element by element: FP32 against FP64 accumulation of each sum
            err = np.abs(got.astype(np.float64) - ref)
            bound = 2e-3 * np.abs(ref).max() + 1e-2 * np.abs(ref)
            assert np.all(err <= bound), (l, float((err / np.maximum(bound, 1e-300)).max()),
                                          np.unravel_index(np.argmax(err - bound), err.shape))


def test_gradients_against_fp64_net(env):
    """The same gradients against the oracle's plain FP64 net (hidden
    activations not rounded): what differs is the BF16 storage of the GPU's
    activations (relative 2^-9 per value, through four layers, and the ReLU
    decisions it moves), measured at up to 6 % of a layer's gradient norm; the
    bound is 10 %, per layer and element by element (each element's error
    against the layer's largest gradient plus its own magnitude).  A wrong
    layer, a transposed or shifted tap would be off by order one."""
    torch, P, O = env
    B, H, W = 2, 24, 90
    rng = np.random.default_rng(321)
    sur = P.Surrogate(seed=12)
    p = sur.params()
    p[:] = rng.normal(0, 1, p.size).astype(np.float32) * np.float32(0.12)
    sur.set_params(p)
    x = _inputs(rng, B, H, W)
    t = rng.normal(0, 0.05, (B, H - 10, W - 10, 3)).astype(np.float32)
    loss, g = sur.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    layers = sur.layers(p)
    ws = [bf16(w).astype(np.float64) for w, _ in layers]
    bs = [b.astype(np.float64) for _, b in layers]
    ws[-1] = ws[-1] * OUT_SCALE
    bs[-1] = bs[-1] * OUT_SCALE
    ref_loss = 0.0
    ref_g = [np.zeros_like(w) for w in ws] + [np.zeros_like(b) for b in bs]
    for b in range(B):
        lb, dws, dbs = O.net_loss_grad(split(x[b]).astype(np.float64), ws, bs, t[b].astype(np.float64),
                                       act_bf16=False)
        ref_loss += lb / B
        for l in range(len(ws)):
            scale = OUT_SCALE if l == len(ws) - 1 else 1.0
            ref_g[l] += scale * dws[l] / B
            ref_g[len(ws) + l] += scale * dbs[l] / B
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss, (loss, ref_loss)
    stats = []
    for l, (dw, db) in enumerate(sur.layers(g)):
        for got, ref in ((dw, ref_g[l]), (db, ref_g[len(ws) + l])):
            rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
            err = np.abs(got.astype(np.float64) - ref)
            elem = float((err / (np.abs(ref).max() + np.abs(ref))).max())
            stats.append((l, round(float(rel), 4), round(elem, 4)))
    print("gradients against the FP64 net (layer, norm-relative, element):", stats)
    for l, rel, elem in stats:
        assert rel <= 0.1 and elem <= 0.1, stats


def test_gradients_deterministic(env):
    torch, P, O = env
    rng = np.random.default_rng(5)
    sur = P.Surrogate(seed=2)
    x = torch.from_numpy(_inputs(rng, 3, 30, 70)).cuda()
    t = torch.from_numpy(rng.normal(0, 0.05, (3, 20, 60, 3)).astype(np.float32)).cuda()
    l1, g1 = sur.gradients(x, t)
    l2, g2 = sur.gradients(x, t)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_training_reduces_loss(env):
    """Adam on a local linear target (five explicit diffusion sweeps of
    (h, hu, hv), a 11 x 11 stencil the net can represent): the loss falls by an
    order of magnitude within 100 steps."""
    torch, P, O = env
    rng = np.random.default_rng(7)
    B, H, W = 4, 40, 40
    x = _inputs(rng, B, H, W)
    u = x[..., :3].astype(np.float64)
    for _ in range(5):
        lap = u[:, :-2, 1:-1] + u[:, 2:, 1:-1] + u[:, 1:-1, :-2] + u[:, 1:-1, 2:] - 4 * u[:, 1:-1, 1:-1]
        u = u[:, 1:-1, 1:-1] + 0.002 * lap
    t = (u - x[:, 5:-5, 5:-5, :3]).astype(np.float32)
    sur = P.Surrogate(seed=0)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = [sur.train_step(xd, td, 2e-3) for _ in range(100)]
    assert np.isfinite(losses).all()
    assert min(losses[-10:]) < 0.1 * losses[0], (losses[0], losses[-10:])


def test_max_ctas_rejects_negative_and_keeps_results(env):
    """fp_surrogate_set_max_ctas: a negative limit is refused; the forward on
    one CTA per kernel gives the same bytes as on all (the forward's sums do
    not depend on how work items are spread over CTAs)."""
    torch, P, O = env
    rng = np.random.default_rng(4)
    sur = P.Surrogate(seed=5)
    with pytest.raises(P.FloodPedError):
        sur.set_max_ctas(-1)
    x = torch.from_numpy(_inputs(rng, 2, 40, 150)).cuda()
    y_all = torch.zeros((2, 30, 140, 3), device="cuda")
    y_one = torch.zeros_like(y_all)
    sur.forward(x, y_all)
    sur.set_max_ctas(1)
    sur.forward(x, y_one)
    torch.cuda.synchronize()
    assert torch.equal(y_all, y_one)
