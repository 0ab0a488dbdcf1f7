"""Pins for the corrector oracle (not GPU): the convolution against a
direct numpy evaluation of its definition and, for one channel, against
scipy's 3-D cross-correlation, GELU against its closed form and
the standard normal CDF, and the whole network's gradient against central
finite differences."""
import math

import numpy as np
import pytest

import oracle


def numpy_conv(x, W, b):
    S, Z, Y, X, Ci = x.shape
    Co = W.shape[1]
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(b, (S, Z, Y, X, Co)).copy()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                sl = xp[:, 1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X, :]
                out += np.einsum("szyxc,oc->szyxo", sl, W[t])
    return out


def test_conv_matches_numpy_definition():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 5, 6, 3))
    W = rng.standard_normal((27, 4, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(oracle.conv3d_fwd(x, W, b), numpy_conv(x, W, b), rtol=1e-12, atol=1e-12)


def test_conv_backward_is_the_adjoint():
    """<conv(x), g> = <x, conv^T(g)> and dW, db are the exact gradients of
    the linear functional <conv(x; W, b), g>."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 3, 4, 5, 2))
    W = rng.standard_normal((27, 3, 2))
    g = rng.standard_normal((1, 3, 4, 5, 3))
    dx, dW, db = oracle.conv3d_bwd(x, W, g)
    lhs = np.sum(oracle.conv3d_fwd(x, W, None) * g)
    assert abs(lhs - np.sum(x * dx)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * dW)) < 1e-10 * abs(lhs)
    np.testing.assert_allclose(db, g.sum(axis=(0, 1, 2, 3)), rtol=1e-13)


def test_gelu_tanh_form():
    """The activation is the tanh form of GELU (Hendrycks and Gimpel 2016).
    Pinned by what holds for it independently of its formula: it is within
    5e-4 of the exact x Phi(x) everywhere (the published approximation's
    maximum deviation is 4.7e-4, near x = -2.7), GELU(x) - GELU(-x) = x (the
    inner function is odd), it tends to x and to 0 in the two tails, and its
    derivative matches a central difference."""
    x = np.linspace(-8, 8, 1601)
    phi = np.array([0.5 * (1 + math.erf(v / math.sqrt(2))) for v in x])
    g = oracle.gelu(x)
    dev = np.abs(g - x * phi)
    assert dev.max() < 5e-4 and dev.max() > 4e-4
    np.testing.assert_allclose(g - oracle.gelu(-x), x, rtol=0, atol=1e-14)
    big = np.array([12.0, -12.0])
    np.testing.assert_allclose(oracle.gelu(big), [12.0, 0.0], atol=1e-12)
    h = 1e-6
    fd = (oracle.gelu(x + h) - oracle.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(oracle.gelu(x, grad=True), fd, rtol=1e-7, atol=1e-9)
    assert oracle.gelu(np.array([0.0]))[0] == 0.0


def test_network_gradient_finite_differences():
    """5-layer network (channels 3-4-4-4-4-3) on a 1x3x3x4 box: every
    parameter's gradient against a central finite difference (rel < 1e-6)."""
    ch = [3, 4, 4, 4, 4, 3]
    rng = np.random.default_rng(2)
    n = oracle.corrector_param_count(ch)
    params = 0.3 * rng.standard_normal(n)
    x = rng.standard_normal((1, 3, 3, 4, 3))
    t = rng.standard_normal((1, 3, 3, 4, 3))
    loss, grad, _ = oracle.corrector_loss(params, ch, x, t)
    h = 1e-5
    idx = rng.choice(n, 60, replace=False)
    for i in idx:
        pp = params.copy()
        pp[i] += h
        lp, _, _ = oracle.corrector_loss(pp, ch, x, t, want_grad=False)
        pp[i] -= 2 * h
        lm, _, _ = oracle.corrector_loss(pp, ch, x, t, want_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, grad[i])


def test_conv_single_channel_is_scipy_correlation():
    """One input and one output channel: the oracle's convolution is the
    library's 3-D cross-correlation with zero padding (scipy.ndimage), tap
    (dz, dy, dx) weighting x(z + dz, y + dy, x + dx). A flipped or
    transposed kernel, or a wrong tap order, fails here (the kernel below
    has no symmetry)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(5)
    x = rng.standard_normal((1, 5, 6, 7, 1))
    w = rng.standard_normal((3, 3, 3))  # w[dz + 1, dy + 1, dx + 1]
    W = w.reshape(27, 1, 1)
    want = ndimage.correlate(x[0, ..., 0], w, mode="constant", cval=0.0)
    got = oracle.conv3d_fwd(x, W, None)[0, ..., 0]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    # and it is not the convolution (the flipped kernel)
    assert not np.allclose(got, ndimage.convolve(x[0, ..., 0], w, mode="constant", cval=0.0))
