"""Learned-corrector kernels (BF16 tcgen05 convolutions, FP32 accumulation)
against the FP64 CPU oracle: every layer's pre-activation output, the loss,
and the parameter gradient of the whole network; and Adam steps that lower
the loss."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

CH_REAL = [24, 32, 32, 32, 32, 24]
NTAP, CH = 27, 32
LAYER = NTAP * CH * CH + CH


def bf16_round(a):
    """Round float64 values to the nearest BF16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def padded_to_oracle(p):
    """GPU packing (5 x (W[27][32][32], b[32])) -> oracle packing with the
    real channel counts 24-32-32-32-32-24."""
    out = []
    for l in range(5):
        W = p[l * LAYER:l * LAYER + NTAP * CH * CH].reshape(NTAP, CH, CH).astype(np.float64)
        b = p[l * LAYER + NTAP * CH * CH:(l + 1) * LAYER].astype(np.float64)
        ci, co = CH_REAL[l], CH_REAL[l + 1]
        out += [W[:, :co, :ci].ravel(), b[:co]]
    return np.concatenate(out)


def seeded_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(5 * LAYER, dtype=np.float32)
    for l in range(5):
        ci, co = CH_REAL[l], CH_REAL[l + 1]
        W = np.zeros((NTAP, CH, CH))
        W[:, :co, :ci] = rng.uniform(-1, 1, (NTAP, co, ci)) * np.sqrt(3.0 / (27 * ci)) * scale
        b = np.zeros(CH)
        b[:co] = rng.uniform(-0.1, 0.1, co)
        p[l * LAYER:(l + 1) * LAYER] = np.concatenate([bf16_round(W).ravel(), b]).astype(np.float32)
    return p


def to_bf16_tensor(x):
    torch = need_gpu()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to("cuda").to(torch.bfloat16)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def net32():
    torch = need_gpu()
    c = B.corrector_create(32, 2, seed=7)
    yield c
    B.corrector_destroy(c)


@pytest.mark.parametrize("S", [1, 2])
def test_every_layer_matches_oracle_conv(net32, S):
    """Pre-activation of each layer against the oracle convolution of that
    layer's BF16 input (the previous layer's GELU output rounded to BF16).
    At 32^3 the work units hold 3 (S = 1) or 6 (S = 2) output planes of 3
    rows, so both leave a short last run of planes and a short last block of
    rows."""
    torch = need_gpu()
    n = 32
    p = seeded_params(11)
    B.corrector_params(net32, p)
    rng = np.random.default_rng(12 + S)
    x = np.zeros((S, n, n, n, CH))
    x[..., :24] = bf16_round(rng.standard_normal((S, n, n, n, 24)))
    out = torch.empty((S * n ** 3, CH), dtype=torch.float32, device="cuda")
    B.corrector_forward_raw(net32, S, to_bf16_tensor(x), out)
    act = x
    for l in range(5):
        z = torch.empty_like(out)
        if l < 4:
            B.corrector_layer_output(net32, l, S, z)
        else:
            z = out  # forward_raw writes the last layer straight into out
        zg = z.cpu().numpy().reshape(S, n, n, n, CH)
        W = p[l * LAYER:l * LAYER + NTAP * CH * CH].reshape(NTAP, CH, CH).astype(np.float64)
        b = p[l * LAYER + NTAP * CH * CH:(l + 1) * LAYER].astype(np.float64)
        want = oracle.conv3d_fwd(act, W, b)
        err = rel(zg, want)
        assert err < 2e-3, (l, err)
        act = bf16_round(oracle.gelu(zg))  # the next layer's input as the GPU forms it


def test_first_layer_at_64_cubed():
    """The 64^3 grid of the learned form: units of 3 rows (two 128-entry
    tiles) and 5 planes, N = 96 stacked MMAs, against the oracle."""
    torch = need_gpu()
    n = 64
    c = B.corrector_create(n, 1, seed=3)
    try:
        p = seeded_params(31)
        B.corrector_params(c, p)
        rng = np.random.default_rng(32)
        x = np.zeros((1, n, n, n, CH))
        x[..., :24] = bf16_round(rng.standard_normal((1, n, n, n, 24)))
        out = torch.empty((n ** 3, CH), dtype=torch.float32, device="cuda")
        B.corrector_forward_raw(c, 1, to_bf16_tensor(x), out)
        z = torch.empty_like(out)
        B.corrector_layer_output(c, 0, 1, z)
        zg = z.cpu().numpy().reshape(1, n, n, n, CH)
        W = p[:NTAP * CH * CH].reshape(NTAP, CH, CH).astype(np.float64)
        b = p[NTAP * CH * CH:LAYER].astype(np.float64)
        want = oracle.conv3d_fwd(x, W, b)
        assert rel(zg, want) < 2e-3
        # every point, not only on average
        assert np.max(np.abs(zg - want)) < 2e-2 * np.max(np.abs(want))
    finally:
        B.corrector_destroy(c)


@pytest.mark.parametrize("n,S", [(32, 2), (64, 1)])
def test_async_inference_is_the_forward_pass(n, S):
    """The serving call (enqueued without a host wait, no hidden
    pre-activations stored) gives the synchronous forward pass's output bit
    for bit, and queued calls on one stream each see their own input."""
    torch = need_gpu()
    c = B.corrector_create(n, S, seed=5)
    try:
        B.corrector_params(c, seeded_params(41))
        rng = np.random.default_rng(42 + n)
        xs = []
        for _ in range(2):
            x = np.zeros((S, n, n, n, CH))
            x[..., :24] = bf16_round(rng.standard_normal((S, n, n, n, 24)))
            xs.append(to_bf16_tensor(x))
        want = []
        for x in xs:
            o = torch.empty((S * n ** 3, CH), dtype=torch.float32, device="cuda")
            B.corrector_forward_raw(c, S, x, o)
            want.append(o)
        got = [torch.full_like(w, float("nan")) for w in want]
        for x, o in zip(xs, got):
            B.corrector_infer_async(c, S, x, o)
        B.corrector_sync(c)
        for g, w in zip(got, want):
            assert torch.equal(g, w)
        assert not torch.equal(got[0], got[1])
    finally:
        B.corrector_destroy(c)


def test_loss_and_gradient_match_oracle(net32):
    torch = need_gpu()
    n, S = 32, 1
    p = seeded_params(21)
    B.corrector_params(net32, p)
    rng = np.random.default_rng(22)
    x = np.zeros((S, n, n, n, CH))
    x[..., :24] = bf16_round(rng.standard_normal((S, n, n, n, 24)))
    t = np.zeros((S, n ** 3, CH), dtype=np.float32)
    t[..., :24] = 0.3 * rng.standard_normal((S, n ** 3, 24))
    loss = B.corrector_loss_grad_raw(net32, S, to_bf16_tensor(x), torch.from_numpy(t).cuda())
    g_gpu = padded_to_oracle(B.corrector_grads(net32))
    want_loss, g_or, _ = oracle.corrector_loss(padded_to_oracle(p), CH_REAL, x[..., :24],
                                               t[..., :24].reshape(S, n, n, n, 24).astype(np.float64))
    assert abs(loss - want_loss) < 1e-2 * want_loss
    cos = np.dot(g_gpu, g_or) / (np.linalg.norm(g_gpu) * np.linalg.norm(g_or))
    assert cos > 0.999, cos
    assert rel(g_gpu, g_or) < 5e-2
    # per layer too
    o = 0
    for l in range(5):
        m = 27 * CH_REAL[l + 1] * CH_REAL[l] + CH_REAL[l + 1]
        gl, ol = g_gpu[o:o + m], g_or[o:o + m]
        assert np.dot(gl, ol) / (np.linalg.norm(gl) * np.linalg.norm(ol)) > 0.995, l
        o += m


def test_adam_steps_lower_the_loss(net32):
    """Ten Adam steps on a fixed synthetic regression problem (target a
    smooth function of the input) lower the loss."""
    torch = need_gpu()
    n, S = 32, 2
    B.corrector_params(net32, seeded_params(31, scale=0.5))
    rng = np.random.default_rng(32)
    grid = B.make_grid(n, ghost=3, dx=0.1)
    coarse, target = [], []
    from paper_1307_6488_gb300 import inputs
    for s in range(S):
        u = inputs.flat_space(n, n, n, 3)
        inputs.smooth_perturbation(u, 3, 0.05, 40 + s, 0.1)
        tgt = u.copy()
        tgt[:, 3:-3, 3:-3, 3:-3] += 0.01 * np.tanh(u[:, 3:-3, 3:-3, 3:-3] - 0.5)
        coarse.append(B.upload(u, grid))
        target.append(B.upload(tgt, grid))
    B.corrector_set_scales(net32, np.zeros(24), np.full(24, 10.0), np.full(24, 100.0))
    losses = [B.corrector_train_step(net32, grid, coarse, target, 2e-3) for _ in range(10)]
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0], losses
