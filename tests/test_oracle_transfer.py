"""Pins for the oracle's 2:1 transfer operators (not GPU): tricubic
prolongation reproduces polynomials of degree <= 3 per axis exactly; the
order-2 restriction (the mean of the 8 children) returns the coarse-centre
value of any linear function exactly and misses a quadratic by its closed-form
second moment; the order-4 restriction (tricubic interpolation at the coarse
centre) is exact on tricubics and misses x^4 by the Lagrange remainder; and
restriction after prolongation round-trips tricubics exactly."""
import numpy as np
import pytest

import oracle


def centres(n, g, h, lo=0.0):
    return lo + (np.arange(-g, n + g) + 0.5) * h


def test_prolong_exact_on_tricubics():
    n, cg, fg, H = 5, 2, 1, 0.3
    xc = centres(n, cg, H)
    xf = centres(2 * n, fg, H / 2)
    rng = np.random.default_rng(0)
    c = np.zeros((24, n + 2 * cg, n + 2 * cg, n + 2 * cg))
    f_want = np.zeros((24, 2 * n + 2 * fg, 2 * n + 2 * fg, 2 * n + 2 * fg))
    for v in range(24):
        a, b, d = rng.standard_normal((3, 4))
        px = lambda x: a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3
        py = lambda y: b[0] + b[1] * y + b[2] * y ** 2 + b[3] * y ** 3
        pz = lambda z: d[0] + d[1] * z + d[2] * z ** 2 + d[3] * z ** 3
        c[v] = pz(xc)[:, None, None] * py(xc)[None, :, None] * px(xc)[None, None, :]
        f_want[v] = pz(xf)[:, None, None] * py(xf)[None, :, None] * px(xf)[None, None, :]
    f = oracle.prolong(c, cg, fg)
    I = (slice(None),) + (slice(fg, -fg),) * 3
    np.testing.assert_allclose(f[I], f_want[I], rtol=1e-11, atol=1e-11)


def test_restrict_exact_on_linear():
    n, fg, cg, H = 4, 2, 1, 0.25
    xf = centres(2 * n, fg, H / 2)
    xc = centres(n, cg, H)
    f = np.zeros((24, 2 * n + 2 * fg, 2 * n + 2 * fg, 2 * n + 2 * fg))
    want = np.zeros((24, n + 2 * cg, n + 2 * cg, n + 2 * cg))
    rng = np.random.default_rng(1)
    for v in range(24):
        a = rng.standard_normal(4)
        f[v] = a[0] + a[1] * xf[None, None, :] + a[2] * xf[None, :, None] + a[3] * xf[:, None, None]
        want[v] = a[0] + a[1] * xc[None, None, :] + a[2] * xc[None, :, None] + a[3] * xc[:, None, None]
    c = oracle.restrict(f, fg, cg, order=2)
    I = (slice(None),) + (slice(cg, -cg),) * 3
    np.testing.assert_allclose(c[I], want[I], rtol=1e-13, atol=1e-13)


def tricubic_fields(n, g, h, seed):
    """24 random products of cubics sampled at the cell centres of an n^3 grid
    with g ghosts, spacing h; returns (fields, the polynomials' coefficients)."""
    x = centres(n, g, h)
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal((24, 3, 4))
    u = np.zeros((24,) + (n + 2 * g,) * 3)
    for v in range(24):
        p = [np.polyval(coef[v, k][::-1], x) for k in range(3)]
        u[v] = p[2][:, None, None] * p[1][None, :, None] * p[0][None, None, :]
    return u, coef


def test_restrict4_exact_on_tricubics():
    n, fg, cg, H = 4, 1, 2, 0.25
    f, coef = tricubic_fields(2 * n, fg, H / 2, 3)
    xc = centres(n, cg, H)
    c = oracle.restrict(f, fg, cg, order=4)
    J = (slice(cg, -cg),) * 3
    for v in range(24):
        p = [np.polyval(coef[v, k][::-1], xc) for k in range(3)]
        want = p[2][:, None, None] * p[1][None, :, None] * p[0][None, None, :]
        np.testing.assert_allclose(c[v][J], want[J], rtol=1e-12, atol=1e-12)


def test_restrict_remainders():
    """x^2 under the 8-child mean: children at x -+ hf/2, mean x^2 + hf^2/4.
    x^4 under 4-point midpoint interpolation: the Lagrange remainder is
    (d^4 f / 4!) prod (x - x_m) = (3/2)(1/2)(1/2)(3/2) hf^4 = 9/16 hf^4, so
    the interpolant is x^4 - 9/16 hf^4."""
    n, fg, cg, hf = 3, 1, 1, 0.2
    xf = centres(2 * n, fg, hf)
    xc = centres(n, cg, 2 * hf)
    J = (slice(cg, -cg),) * 3
    f = np.broadcast_to(xf[None, None, None, :] ** 2, (24,) + (2 * n + 2 * fg,) * 3).copy()
    c = oracle.restrict(f, fg, cg, order=2)
    want = np.broadcast_to(xc[None, None, :] ** 2 + hf ** 2 / 4, (n + 2 * cg,) * 3)
    np.testing.assert_allclose(c[0][J], want[J], rtol=1e-14, atol=1e-15)
    f = np.broadcast_to(xf[None, None, None, :] ** 4, (24,) + (2 * n + 2 * fg,) * 3).copy()
    c = oracle.restrict(f, fg, cg, order=4)
    want = np.broadcast_to(xc[None, None, :] ** 4 - 9.0 / 16.0 * hf ** 4, (n + 2 * cg,) * 3)
    np.testing.assert_allclose(c[0][J], want[J], rtol=1e-13, atol=1e-14)


def test_restrict4_after_prolong_round_trips_tricubics():
    n, cg, fg, H = 5, 2, 1, 0.3
    c0, _ = tricubic_fields(n, cg, H, 4)
    f = oracle.prolong(c0, cg, fg)
    # the fine interior is the same tricubic; its ghosts come from the
    # polynomial itself (prolongation fills the interior only)
    fx, _ = tricubic_fields(2 * n, fg, H / 2, 4)
    fI = (slice(None),) + (slice(fg, -fg),) * 3
    np.testing.assert_allclose(f[fI], fx[fI], rtol=1e-11, atol=1e-11)
    f[:, :fg], f[:, -fg:] = fx[:, :fg], fx[:, -fg:]
    f[:, :, :fg], f[:, :, -fg:] = fx[:, :, :fg], fx[:, :, -fg:]
    f[:, :, :, :fg], f[:, :, :, -fg:] = fx[:, :, :, :fg], fx[:, :, :, -fg:]
    c = oracle.restrict(f, fg, cg, order=4)
    I = (slice(None),) + (slice(cg, -cg),) * 3
    np.testing.assert_allclose(c[I], c0[I], rtol=1e-11, atol=1e-11)


def test_restrict_rejects_bad_arguments():
    f = np.zeros((24, 8, 8, 8))
    with pytest.raises(ValueError):
        oracle.restrict(f, 0, 1, order=4)  # order 4 needs a fine ghost
    with pytest.raises(ValueError):
        oracle.restrict(f, 1, 1, order=3)
