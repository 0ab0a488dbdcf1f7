"""Pins for the oracle's finite-difference operators (not GPU).

The stencils follow the paper's 'customized finite differencing operators'
(Sec. 2.3) at the orders used for the BSSN run (8th order, Sec. 3.3) and
4th order; their weights are checked against
  * the closed-form textbook weights (Fornberg, Math. Comp. 51 (1988) 699,
    Table 1),
  * numpy's linear solve of the Vandermonde (moment) system,
  * exactness on monomials up to the operator's degree,
and Kreiss-Oliger dissipation against its closed-form Fourier symbol.
"""
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle



def _textbook():
    """Closed-form centred weights w_a, a = 1..p/2, from the golden table
    (Fornberg 1988, Table 1): {(m, order): [w_1, w_2, ...]}."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fd_weights.txt")
    table = {}
    for m, order, a, num, den in np.loadtxt(path, comments="#", dtype=np.int64):
        table.setdefault((int(m), int(order)), {})[int(a)] = F(int(num), int(den))
    return {k: [v[a] for a in sorted(v)] for k, v in table.items()}


TEXTBOOK = _textbook()


@pytest.mark.parametrize("m,order", [(1, 4), (1, 8), (2, 4), (2, 8)])
def test_centered_weights_textbook(m, order):
    half = order // 2
    offs = list(range(-half, half + 1))
    for a in range(1, half + 1):
        num, den = oracle.fd_weight(offs, m, half + a)
        assert F(num, den) == TEXTBOOK[(m, order)][a - 1]
    st = oracle.stencils(order)
    key = "c1" if m == 1 else "c2"
    np.testing.assert_array_equal(st[key], [float(w) for w in TEXTBOOK[(m, order)]])
    if m == 2:
        # centre weight of the second derivative is -2 sum(w_a)
        num, den = oracle.fd_weight(offs, 2, half)
        assert F(num, den) == -2 * sum(TEXTBOOK[(2, order)])


def test_upwind_4th_textbook():
    # (-3 u_-1 - 10 u_0 + 18 u_1 - 6 u_2 + u_3) / 12
    st = oracle.stencils(4)
    assert st["up_lo"] == -1
    np.testing.assert_allclose(st["up"], np.array([-3, -10, 18, -6, 1]) / 12.0, rtol=0, atol=1e-16)


@pytest.mark.parametrize("order", [4, 8])
def test_weights_match_vandermonde_solve(order):
    st = oracle.stencils(order)
    half = order // 2
    for m, key in ((1, "c1"), (2, "c2")):
        offs = np.arange(-half, half + 1, dtype=np.float64)
        V = np.vander(offs, increasing=True).T  # V[q, j] = o_j^q
        rhs = np.zeros(len(offs))
        rhs[m] = float(np.prod(np.arange(1, m + 1)))
        w = np.linalg.solve(V, rhs)
        np.testing.assert_allclose(st[key], w[half + 1:], rtol=1e-11, atol=1e-13)
    offs = np.arange(st["up_lo"], st["up_lo"] + len(st["up"]), dtype=np.float64)
    V = np.vander(offs, increasing=True).T
    rhs = np.zeros(len(offs))
    rhs[1] = 1.0
    np.testing.assert_allclose(st["up"], np.linalg.solve(V, rhs), rtol=1e-10, atol=1e-12)
    r = st["r"]
    assert r == half + 1
    # Kreiss-Oliger: (2r)-th undivided difference = binomial weights with
    # alternating sign
    from math import comb
    np.testing.assert_array_equal(st["ko"], [(-1) ** (a + r) * comb(2 * r, r + a) for a in range(-r, r + 1)])


def _grid(n, g, h, lo=(-0.3, 0.2, 0.1)):
    xs = [lo[a] + (np.arange(-g, n + g) + 0.5) * h for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z


@pytest.mark.parametrize("order", [4, 8])
def test_polynomial_exactness(order):
    g = order // 2 + 1
    n, h = 5, 0.13
    X, Y, Z = _grid(n, g, h)
    I = (slice(g, g + n),) * 3
    C = (X, Y, Z)
    p = order
    rng = np.random.default_rng(7)
    # first derivatives: exact up to degree p; second: up to p+1;
    # mixed: x^a y^b with a, b <= p; upwind: degree p.
    for deg in range(0, p + 1):
        for axis in range(3):
            coef = rng.uniform(0.5, 1.5)
            u = coef * C[axis] ** deg
            du = coef * deg * C[axis] ** max(deg - 1, 0) if deg > 0 else 0 * u
            out = oracle.apply_op(u, g, h, order, 0, a=axis)
            scale = np.max(np.abs(u[I])) / h + 1
            assert np.max(np.abs(out[I] - du[I])) < 1e-12 * scale, (deg, axis)
            for beta in (0.7, -0.4):
                out = oracle.apply_op(u, g, h, order, 3, a=axis, beta=beta)
                assert np.max(np.abs(out[I] - beta * du[I])) < 1e-12 * scale, (deg, axis, beta)
    for deg in range(0, p + 2):
        for axis in range(3):
            u = C[axis] ** deg
            d2 = deg * (deg - 1) * C[axis] ** max(deg - 2, 0) if deg > 1 else 0 * u
            out = oracle.apply_op(u, g, h, order, 1, a=axis)
            scale = np.max(np.abs(u[I])) / h ** 2 + 1
            assert np.max(np.abs(out[I] - d2[I])) < 1e-12 * scale, (deg, axis)
    for da in range(0, p + 1, 2):
        for db in range(1, p + 1, 3):
            for (a, b) in ((0, 1), (0, 2), (1, 2)):
                u = C[a] ** da * C[b] ** db
                exact = (da * C[a] ** max(da - 1, 0) if da else 0 * u) * (db * C[b] ** max(db - 1, 0))
                out = oracle.apply_op(u, g, h, order, 2, a=a, b=b)
                scale = np.max(np.abs(u[I])) / h ** 2 + 1
                assert np.max(np.abs(out[I] - exact[I])) < 1e-12 * scale, (da, db, a, b)
    # KO annihilates polynomials of degree < 2r in every direction
    r = order // 2 + 1
    for deg in range(0, 2 * r):
        u = X ** deg + Y ** (deg // 2) * Z ** (deg - deg // 2)
        out = oracle.apply_op(u, g, h, order, 4, beta=0.1)
        assert np.max(np.abs(out[I])) < 1e-12 * (np.max(np.abs(u[I])) / h + 1)
    # ... and the first-derivative stencil is not exact one degree higher
    u = X ** (p + 1)
    out = oracle.apply_op(u, g, h, order, 0, a=0)
    assert np.max(np.abs(out[I] - (p + 1) * X[I] ** p)) > 1e-10


@pytest.mark.parametrize("order", [4, 8])
def test_ko_fourier_symbol(order):
    """delta^(2r) e^{ikx} = (-4 sin^2(kh/2))^r e^{ikx}, so the dissipation
    operator maps sin(kx) to -(eps/h) sin^(2r)(kh/2) sin(kx) per direction."""
    g = order // 2 + 1
    n, h, eps = 12, 1.0 / 12, 0.1
    X, Y, Z = _grid(n, g, h, lo=(0, 0, 0))
    I = (slice(g, g + n),) * 3
    r = order // 2 + 1
    for kx, ky in ((2, 0), (3, 5)):
        k1, k2 = 2 * np.pi * kx, 2 * np.pi * ky
        u = np.sin(k1 * X) + np.sin(k2 * Y)
        out = oracle.apply_op(u, g, h, order, 4, beta=eps)
        exact = -(eps / h) * (np.sin(k1 * h / 2) ** (2 * r) * np.sin(k1 * X) + np.sin(k2 * h / 2) ** (2 * r) * np.sin(k2 * Y))
        np.testing.assert_allclose(out[I], exact[I], rtol=0, atol=1e-12)


@pytest.mark.parametrize("order", [4, 8])
def test_mixed_derivative_accurate_under_one_axis_variation(order):
    """Data varying by 1e-2 along x but only by 1e-10 along y: the oracle's
    mixed derivative agrees with the exact rational evaluation of the same
    tensor-product stencil on the same stored doubles to 1e-12 relative.
    Differences of stored values are taken before any weight is applied, so
    they are exact; applying the rounded first-derivative stencil first and
    then differencing its outputs misses by about 4e-7 relative here at 8th
    order."""
    g = order // 2 + 1
    n, h = 4, 1.0 / 24
    X, Y, Z = _grid(n, g, h)
    u = 1 + 0.01 * np.sin(2 * np.pi * X) + 1e-10 * np.cos(2 * np.pi * (X + 2 * Y))
    out = oracle.apply_op(u, g, h, order, 2, a=0, b=1)
    w = [F(x) for x in TEXTBOOK[(1, order)]]
    hf = F(h)
    half = order // 2
    for (k, j, i) in ((g, g, g), (g + 1, g + 2, g + 3), (g + 3, g + 1, g)):
        ex = F(0)
        for a in range(1, half + 1):
            for b in range(1, half + 1):
                q = (F(u[k, j + b, i + a]) - F(u[k, j + b, i - a])) - (F(u[k, j - b, i + a]) - F(u[k, j - b, i - a]))
                ex += w[a - 1] * w[b - 1] * q
        ex = ex / (hf * hf)
        assert abs(F(out[k, j, i]) - ex) <= F(1, 10 ** 12) * abs(ex)
