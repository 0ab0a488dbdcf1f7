"""Pins for the oracle's RK4 step, ghost filling and dissipation (not GPU).

The paper integrates with a Runge-Kutta method of lines (Sec. 3.3, RK3);
this build uses the classic four-stage RK4. Pins:
  * a linear homogeneous system (Gamma-driver shift, constant fields): one
    RK4 step applies exactly the degree-4 Taylor polynomial of exp(dt M);
  * homogeneous harmonic slicing has a closed-form lapse and K, and
    homogeneous 1+log slicing a conserved combination of them; RK4 meets
    both at 4th order in dt;
  * periodic and static ghost filling match their definitions.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import inputs
from paper_1307_6488_gb300.inputs import IDX, NVAR


def homogeneous(g, n=4, **vals):
    u = inputs.flat_space(n, n, n, g)
    for k, v in vals.items():
        u[IDX[k]] = v
    return u


@pytest.mark.parametrize("order", [4, 8])
def test_rk4_linear_gamma_driver(order):
    g = order // 2 + 1
    b0 = np.array([0.3, -0.2, 0.11])
    B0 = np.array([0.05, 0.07, -0.09])
    u = homogeneous(g, beta1=b0[0], beta2=b0[1], beta3=b0[2], B1=B0[0], B2=B0[1], B3=B0[2])
    eta, c, dt = 2.0, 0.75, 0.05
    p = oracle.Params(fd_order=order, lapse=2, shift=0, eta=eta, shift_coeff=c)
    y = oracle.rk4_step(u, g, 0.1, dt, p, bc=0)
    z = -eta * dt
    P = sum(z ** k / math.factorial(k) for k in range(5))
    S = sum(z ** (k - 1) / math.factorial(k) for k in range(1, 5))
    for i in range(3):
        np.testing.assert_allclose(y[IDX["B1"] + i], B0[i] * P, rtol=1e-14, atol=1e-17)
        np.testing.assert_allclose(y[IDX["beta1"] + i], b0[i] + c * dt * B0[i] * S, rtol=1e-14, atol=1e-17)


def _evolve_homogeneous(lapse, a0, K0, T, nsteps):
    g = 3
    p = oracle.Params(fd_order=4, lapse=lapse, shift=1)
    u = homogeneous(g, alpha=a0, trK=K0)
    for _ in range(nsteps):
        u = oracle.rk4_step(u, g, 0.1, T / nsteps, p, bc=0)
    return u[IDX["alpha"], g, g, g], u[IDX["trK"], g, g, g]


def test_rk4_harmonic_closed_form():
    """Homogeneous data with harmonic slicing: alpha' = -alpha^2 K,
    K' = alpha K^2/3 integrate to alpha = alpha0 (1 + 2 K0 alpha0 t/3)^(-3/2),
    K = K0 (1 + 2 K0 alpha0 t/3)^(1/2); RK4 converges to it at 4th order."""
    a0, K0, T = 0.9, 0.4, 0.5
    s = 1 + 2 * K0 * a0 * T / 3
    a_ex, K_ex = a0 * s ** -1.5, K0 * s ** 0.5
    errs = []
    for n in (5, 10, 20):
        a, K = _evolve_homogeneous(1, a0, K0, T, n)
        errs.append(max(abs(a - a_ex), abs(K - K_ex)))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 3.7 < r1 < 4.4 and 3.7 < r2 < 4.4, errs


def test_rk4_one_plus_log_invariant():
    """Homogeneous data with 1+log slicing: alpha' = -2 alpha K and
    K' = alpha K^2/3 give dK/dalpha = -K/6, so K exp((alpha - alpha0)/6)
    stays K0; RK4 conserves it to 4th order in dt."""
    a0, K0, T = 0.9, 0.4, 0.5
    errs = []
    for n in (5, 10, 20):
        a, K = _evolve_homogeneous(0, a0, K0, T, n)
        assert abs(a - a0) > 0.1  # the lapse really evolved
        errs.append(abs(K * np.exp((a - a0) / 6) - K0))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 3.7 < r1 < 4.4 and 3.7 < r2 < 4.4, errs


def test_periodic_fill():
    g, n = 3, 5
    rng = np.random.default_rng(3)
    u = rng.standard_normal((NVAR, n + 2 * g, n + 2 * g, n + 2 * g))
    ref = u.copy()
    oracle.fill_ghosts(u, g, mode=0)
    idx = (np.arange(-g, n + g) % n) + g
    want = ref[:, idx][:, :, idx][:, :, :, idx]
    np.testing.assert_array_equal(u, want)


def test_static_fill():
    g, n = 2, 4
    rng = np.random.default_rng(4)
    u = rng.standard_normal((NVAR, n + 2 * g, n + 2 * g, n + 2 * g))
    src = rng.standard_normal(u.shape)
    ref = u.copy()
    oracle.fill_ghosts(u, g, mode=1, src=src)
    mask = np.ones(u.shape[1:], dtype=bool)
    mask[g:g + n, g:g + n, g:g + n] = False
    assert np.array_equal(u[:, mask], src[:, mask])
    assert np.array_equal(u[:, ~mask], ref[:, ~mask])


def test_rk4_step_matches_stagewise_definition():
    """The RK4 step equals y0 + dt/6 (k1 + 2k2 + 2k3 + k4) built from the
    oracle's own f = RHS + KO with ghosts filled before every stage."""
    g = 3
    u, h = inputs.gauge_wave(6, g, amplitude=0.05, noise=1e-3, seed=5)
    p = oracle.Params(fd_order=4)
    dt = 0.25 * h

    def f(y):
        y = oracle.fill_ghosts(y.copy(), g, 0)
        return oracle.rhs(y, g, h, p, ko=True)

    k1 = f(u)
    k2 = f(u + dt / 2 * k1)
    k3 = f(u + dt / 2 * k2)
    k4 = f(u + dt * k3)
    want = oracle.fill_ghosts(u + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4), g, 0)
    got = oracle.rk4_step(u, g, h, dt, p, bc=0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
