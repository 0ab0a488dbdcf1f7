"""Pins for the oracle's third-order Runge-Kutta step (not GPU).

The paper integrates with a third-order Runge-Kutta method of lines
(Sec. 3.3). The oracle takes it as the strong-stability-preserving method of
Shu & Osher (1988) in its convex-combination form. Pins:
  * the same method written as a Butcher tableau (c = 0, 1, 1/2;
    a21 = 1, a31 = a32 = 1/4; b = 1/6, 1/6, 2/3) from the oracle's own
    f = RHS + KO gives the same step;
  * on a linear homogeneous system (Gamma-driver shift, constant fields)
    one step applies exactly the degree-3 Taylor polynomial of exp(dt M);
  * homogeneous harmonic slicing (closed form) and homogeneous 1+log slicing
    (conserved K exp((alpha - alpha0)/6)) are met at 3rd order in dt.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import inputs
from paper_1307_6488_gb300.inputs import IDX


def homogeneous(g, n=4, **vals):
    u = inputs.flat_space(n, n, n, g)
    for k, v in vals.items():
        u[IDX[k]] = v
    return u


def test_rk3_matches_butcher_form():
    g = 3
    u, h = inputs.gauge_wave(6, g, amplitude=0.05, noise=1e-3, seed=5)
    p = oracle.Params(fd_order=4)
    dt = 0.25 * h

    def f(y):
        y = oracle.fill_ghosts(y.copy(), g, 0)
        return oracle.rhs(y, g, h, p, ko=True)

    k1 = f(u)
    k2 = f(u + dt * k1)
    k3 = f(u + dt / 4 * (k1 + k2))
    want = oracle.fill_ghosts(u + dt * (k1 / 6 + k2 / 6 + 2 * k3 / 3), g, 0)
    got = oracle.rk3_step(u, g, h, dt, p, bc=0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("order", [4, 8])
def test_rk3_linear_gamma_driver(order):
    g = order // 2 + 1
    b0 = np.array([0.3, -0.2, 0.11])
    B0 = np.array([0.05, 0.07, -0.09])
    u = homogeneous(g, beta1=b0[0], beta2=b0[1], beta3=b0[2], B1=B0[0], B2=B0[1], B3=B0[2])
    eta, c, dt = 2.0, 0.75, 0.05
    p = oracle.Params(fd_order=order, lapse=2, shift=0, eta=eta, shift_coeff=c)
    y = oracle.rk3_step(u, g, 0.1, dt, p, bc=0)
    z = -eta * dt
    P = sum(z ** k / math.factorial(k) for k in range(4))
    S = sum(z ** (k - 1) / math.factorial(k) for k in range(1, 4))
    for i in range(3):
        np.testing.assert_allclose(y[IDX["B1"] + i], B0[i] * P, rtol=1e-14, atol=1e-17)
        np.testing.assert_allclose(y[IDX["beta1"] + i], b0[i] + c * dt * B0[i] * S, rtol=1e-14, atol=1e-17)


def _evolve_homogeneous(lapse, a0, K0, T, nsteps):
    g = 3
    p = oracle.Params(fd_order=4, lapse=lapse, shift=1)
    u = homogeneous(g, alpha=a0, trK=K0)
    for _ in range(nsteps):
        u = oracle.rk3_step(u, g, 0.1, T / nsteps, p, bc=0)
    return u[IDX["alpha"], g, g, g], u[IDX["trK"], g, g, g]


def test_rk3_harmonic_closed_form():
    a0, K0, T = 0.9, 0.4, 0.5
    s = 1 + 2 * K0 * a0 * T / 3
    a_ex, K_ex = a0 * s ** -1.5, K0 * s ** 0.5
    errs = []
    for n in (5, 10, 20):
        a, K = _evolve_homogeneous(1, a0, K0, T, n)
        errs.append(max(abs(a - a_ex), abs(K - K_ex)))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 2.7 < r1 < 3.4 and 2.7 < r2 < 3.4, errs


def test_rk3_one_plus_log_invariant():
    a0, K0, T = 0.9, 0.4, 0.5
    errs = []
    for n in (5, 10, 20):
        a, K = _evolve_homogeneous(0, a0, K0, T, n)
        assert abs(a - a0) > 0.1
        errs.append(abs(K * np.exp((a - a0) / 6) - K0))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 2.7 < r1 < 3.4 and 2.7 < r2 < 3.4, errs
