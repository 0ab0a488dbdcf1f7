"""Pins for the oracle's BSSN right-hand side and constraints (not GPU).

The paper evolves the Einstein equations in BSSN form (Sec. 1.1; 8th-order
finite differences, Sec. 3.3) without writing them out. Each test below
checks the oracle against a property that physics or mathematics fixes,
independently of how the oracle transcribes the equations:

  * flat space has an exactly zero right-hand side;
  * Kasner (homogeneous vacuum, rotated axes): the right-hand side equals
    the exact time derivative of the BSSN variables to rounding;
  * the gauge wave (harmonic slicing): right-hand side -> exact d/dt at the
    stencil order;
  * Kerr-Schild and isotropic Schwarzschild (stationary, frozen gauge):
    right-hand side -> 0 at the stencil order, constraints -> 0;
  * conformally flat York data: momentum constraint -> 0 and Hamiltonian
    constraint -> its closed form at the stencil order;
  * Brill-Lindquist: momentum constraint and several right-hand sides are
    exactly zero;
  * relabelling the axes permutes the right-hand side accordingly;
  * reflecting one axis reflects the right-hand side, each component
    signed by its parity under the reflection.
"""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import inputs
from paper_1307_6488_gb300.inputs import IDX, NVAR

import exact

FROZEN = dict(lapse=2, shift=1)


def interior(a, g):
    return a[..., g:-g, g:-g, g:-g]


def rate(e1, e2):
    return np.log2(e1 / e2)


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("lapse,shift", [(0, 0), (1, 0), (2, 1)])
def test_flat_space_rhs_exactly_zero(order, lapse, shift):
    g = order // 2 + 1
    u = inputs.flat_space(7, 6, 5, g)
    p = oracle.Params(fd_order=order, lapse=lapse, shift=shift)
    r = oracle.rhs(u, g, 0.1, p, ko=True)
    assert np.all(r == 0.0)
    l2, mx, st = oracle.constraints(u, g, 0.1, order)
    assert st == 0 and np.all(l2 == 0.0) and np.all(mx == 0.0)


@pytest.mark.parametrize("order", [4, 8])
def test_flat_space_uniform_shift(order):
    """With a uniform shift every derivative still vanishes; the one-sided
    advection stencil is not in paired form, so the result is zero to
    rounding rather than bitwise."""
    g = order // 2 + 1
    u = inputs.flat_space(6, 6, 6, g, beta=(0.3, -0.2, 0.45))
    p = oracle.Params(fd_order=order)
    r = oracle.rhs(u, g, 0.1, p, ko=True)
    assert np.max(np.abs(r)) < 1e-13


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("pu,angles", [(1.5, (0.3, -0.7, 1.1)), (0.4, (1.2, 0.2, -0.5))])
def test_kasner_exact_time_derivative(order, pu, angles):
    u0, du, _ = exact.kasner(p_u=pu, t0=1.3, angles=angles)
    g = order // 2 + 1
    u = np.broadcast_to(u0[:, None, None, None], (NVAR, 5 + 2 * g, 5 + 2 * g, 5 + 2 * g)).copy()
    p = oracle.Params(fd_order=order, **FROZEN)
    r = oracle.rhs(u, g, 0.1, p, ko=True)
    got = interior(r, g).reshape(NVAR, -1)
    assert np.max(np.abs(got - du[:, None])) < 2e-14
    # Kasner satisfies both constraints
    l2, mx, st = oracle.constraints(u, g, 0.1, order)
    assert np.max(mx[:4]) < 1e-14


def _gw_error(n, order):
    g = order // 2 + 1
    u, h = inputs.gauge_wave(n, g, noise=0.0, ny=g, nz=g)
    p = oracle.Params(fd_order=order, lapse=1, shift=1)
    r = oracle.rhs(u, g, h, p)
    x = -0.5 + (np.arange(-g, n + g) + 0.5) * h
    Xm = np.broadcast_to(x[None, None, :], u.shape[1:])
    dt = exact.gauge_wave_dt(Xm)
    err = np.max(np.abs(interior(r - dt, g)))
    l2, mx, st = oracle.constraints(u, g, h, order)
    return err, mx


@pytest.mark.parametrize("order,ns,lo_rate", [(4, (16, 32, 64), 3.7), (8, (16, 24, 32), 7.5)])
def test_gauge_wave_convergence(order, ns, lo_rate):
    e = [_gw_error(n, order) for n in ns]
    errs = [x[0] for x in e]
    for a in range(len(ns) - 1):
        rr = np.log(errs[a] / errs[a + 1]) / np.log(ns[a + 1] / ns[a])
        assert lo_rate < rr < order + 0.7, (errs, rr)
    # constraints converge to zero at the same order
    for q in range(7):
        c = [x[1][q] for x in e]
        if c[0] > 1e-12:
            rr = np.log(c[0] / c[-1]) / np.log(ns[-1] / ns[0])
            assert rr > lo_rate - 0.5, (q, c)


def _stationary_error(make, n, order, lo, ext, M=1.0):
    g = order // 2 + 1
    h = ext / n
    X, Y, Z = exact.box(n, n, n, g, lo, h)
    u = make(X, Y, Z, M)
    p = oracle.Params(fd_order=order, **FROZEN)
    r = oracle.rhs(u, g, h, p)
    per_var = np.max(np.abs(interior(r, g)).reshape(NVAR, -1), axis=1)
    l2, mx, st = oracle.constraints(u, g, h, order)
    return per_var, mx


STATIONARY = [(4, (12, 24, 48), 3.6, 1.0), (8, (12, 16, 20), 6.5, 2.0)]


@pytest.mark.parametrize("order,ns,lo_rate,ext", STATIONARY)
def test_kerr_schild_stationary(order, ns, lo_rate, ext):
    """Schwarzschild in Kerr-Schild form with its own lapse and shift frozen
    is an exact stationary solution: every right-hand side (including the
    shift, Lie-derivative and Gamma terms) and every constraint -> 0."""
    lo = (1.0, 1.5, 2.0)
    e = [_stationary_error(exact.kerr_schild, n, order, lo, ext) for n in ns]
    for v in range(NVAR):
        errs = [x[0][v] for x in e]
        if v in (IDX["alpha"], IDX["beta1"], IDX["beta2"], IDX["beta3"], IDX["B1"], IDX["B2"], IDX["B3"]):
            assert max(errs) == 0.0
            continue
        rr = np.log(errs[0] / errs[-1]) / np.log(ns[-1] / ns[0])
        assert rr > lo_rate, (inputs.VARS[v], errs, rr)
    for q in range(7):
        c = [x[1][q] for x in e]
        rr = np.log(c[0] / c[-1]) / np.log(ns[-1] / ns[0])
        assert rr > lo_rate, (q, c, rr)


@pytest.mark.parametrize("order,ns,lo_rate,ext", STATIONARY)
def test_isotropic_schwarzschild_static(order, ns, lo_rate, ext):
    """Static Schwarzschild in isotropic coordinates with frozen lapse:
    D^2 alpha = 0 and (-D_i D_j alpha + alpha R_ij)^TF = 0, so the K and
    At right-hand sides converge to zero; the rest are exactly zero."""
    lo = (0.6, 0.9, 1.2)
    e = [_stationary_error(exact.isotropic_schwarzschild, n, order, lo, ext) for n in ns]
    for v in range(NVAR):
        errs = [x[0][v] for x in e]
        if max(errs) == 0.0:
            continue
        assert v in (IDX["trK"],) + tuple(range(IDX["At11"], IDX["At33"] + 1)), inputs.VARS[v]
        rr = np.log(errs[0] / errs[-1]) / np.log(ns[-1] / ns[0])
        assert rr > lo_rate, (inputs.VARS[v], errs, rr)
    c = [x[1][0] for x in e]
    assert np.log(c[0] / c[-1]) / np.log(ns[-1] / ns[0]) > lo_rate


@pytest.mark.parametrize("order,ns,lo_rate", [(4, (12, 24, 48), 3.6), (8, (12, 16, 20), 6.5)])
def test_york_momentum_and_hamiltonian(order, ns, lo_rate):
    g = order // 2 + 1
    errs_m, errs_h = [], []
    for n in ns:
        h = 2.0 / n
        X, Y, Z = exact.box(n, n, n, g, (-1.0, -1.0, -1.0), h)
        u, Hex = exact.momentum_data(X, Y, Z)
        l2, mx, st, (ham, mom, gcon) = oracle.constraints(u, g, h, order, fields=True)
        errs_m.append(max(mx[1:4]))
        errs_h.append(np.max(np.abs(interior(ham - Hex, g))))
        assert np.max(mx[4:]) == 0.0  # gt = delta: Gt_d = 0 = Gt exactly
    for errs in (errs_m, errs_h):
        rr = np.log(errs[0] / errs[-1]) / np.log(ns[-1] / ns[0])
        assert rr > lo_rate, (errs, rr)


def test_brill_lindquist_exact_zeros():
    g = 5
    u, h = inputs.brill_lindquist(16, g)
    p = oracle.Params(fd_order=8)
    r = oracle.rhs(u, g, h, p)
    ri = interior(r, g)
    for name in ["W", "gt11", "gt12", "gt13", "gt22", "gt23", "gt33", "alpha", "beta1", "beta2", "beta3"]:
        assert np.all(ri[IDX[name]] == 0.0), name
    l2, mx, st = oracle.constraints(u, g, h, 8)
    assert st == 0
    assert np.all(mx[1:4] == 0.0)
    assert mx[0] > 0  # punctures make H nonzero near them


@pytest.mark.parametrize("order", [4, 8])
def test_axis_relabelling(order):
    """Cyclically relabelling (x, y, z) -> (y, z, x) maps the right-hand side
    of the relabelled state to the relabelled right-hand side."""
    g = order // 2 + 1
    n = 7
    u, h = inputs.brill_lindquist(n, g, lo=-2.0, hi=2.0, centers=((-0.43, 0.31, 0.2), (0.52, -0.15, -0.33)),
                                  masses=(0.3, 0.4))
    inputs.smooth_perturbation(u, g, 1e-2, 11, h)
    p = oracle.Params(fd_order=order, eta=1.5)
    r = oracle.rhs(u, g, h, p, ko=True)

    perm = [1, 2, 0]  # new axis a is old axis perm[a]

    def relabel(s):
        out = np.empty_like(s)
        # array axes are (z, y, x): new (z', y', x') = old (x, z, y)
        t = np.transpose(s, (0, 3, 1, 2))
        for v in range(NVAR):
            out[v] = t[v]
        res = out.copy()
        # tensor components: new component a <- old component perm[a]
        res[IDX["W"]] = out[IDX["W"]]
        for i in range(3):
            for j in range(i, 3):
                oi, oj = sorted((perm[i], perm[j]))
                res[IDX["gt11"] + inputs.SYM[i][j]] = out[IDX["gt11"] + inputs.SYM[oi][oj]]
                res[IDX["At11"] + inputs.SYM[i][j]] = out[IDX["At11"] + inputs.SYM[oi][oj]]
            for base in ("Gt1", "beta1", "B1"):
                res[IDX[base] + i] = out[IDX[base] + perm[i]]
        return res

    u2 = relabel(u)
    r2 = oracle.rhs(np.ascontiguousarray(u2), g, h, p, ko=True)
    want = relabel(r)
    scale = np.max(np.abs(interior(want, g)).reshape(NVAR, -1), axis=1) + 1e-300
    err = np.max(np.abs(interior(r2 - want, g)).reshape(NVAR, -1), axis=1) / scale
    assert np.max(err) < 1e-13, err


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_reflection(order, axis):
    """Reflecting one coordinate, x_a -> -x_a, maps the right-hand side of the
    reflected state to the reflected right-hand side: each component picks up
    (-1)^(number of indices equal to a). With a generic shift of both signs
    this pins the mirroring of the one-sided advection stencil and every
    sign in the algebra that a relabelling cannot reach."""
    g = order // 2 + 1
    n = 7
    u, h = inputs.brill_lindquist(n, g, lo=-2.0, hi=2.0, centers=((-0.43, 0.31, 0.2), (0.52, -0.15, -0.33)),
                                  masses=(0.3, 0.4))
    inputs.smooth_perturbation(u, g, 3e-2, 17 + axis, h)
    p = oracle.Params(fd_order=order, eta=1.5)
    r = oracle.rhs(u, g, h, p, ko=True)
    sign = np.ones(NVAR)
    for i in range(3):
        for j in range(i, 3):
            s = (-1.0) ** ((i == axis) + (j == axis))
            sign[IDX["gt11"] + inputs.SYM[i][j]] = s
            sign[IDX["At11"] + inputs.SYM[i][j]] = s
    for base in ("Gt1", "beta1", "B1"):
        sign[IDX[base] + axis] = -1.0

    def reflect(s):
        # array axes are (var, z, y, x): coordinate a is array axis 3 - a
        return np.ascontiguousarray(np.flip(s, axis=3 - axis) * sign[:, None, None, None])

    r2 = oracle.rhs(reflect(u), g, h, p, ko=True)
    want = reflect(r)
    scale = np.max(np.abs(interior(want, g)).reshape(NVAR, -1), axis=1) + 1e-300
    err = np.max(np.abs(interior(r2 - want, g)).reshape(NVAR, -1), axis=1) / scale
    assert np.max(err) < 1e-13, dict(zip(inputs.VARS, err))
    # the shift really has both signs along the reflected axis
    b = interior(u, g)[IDX["beta1"] + axis]
    assert b.min() < 0 < b.max()
