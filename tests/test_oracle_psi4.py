"""Pins for the oracle's Weyl diagnostics (not GPU): E_ij, B_ij, Psi_4 and
the invariant I = Q_ij Q^ij / 2, Q = E - i B (the gravitational-wave
extraction the paper runs on the GPU, Sec. 3.3 WeylScal4). Pins:
  * flat space: every output is exactly zero;
  * Kasner (spatially homogeneous, K != 0, zero spatial curvature): the
    eigenvalues of E^i_j are (p_i - p_i^2) / t^2 and B = 0, to rounding;
  * static Schwarzschild in isotropic coordinates (K = 0): B = 0 exactly,
    E_rr (radial unit vector x / (r psi^2)) -> -2M/R^3 with R = r psi^2 the
    areal radius, I -> 3 M^2 / R^6, Psi_4 -> 0 (spherical symmetry: the
    triad is the principal frame), all at the stencils' order;
  * Schwarzschild in Kerr-Schild coordinates (K != 0, shift): the same with
    R the Kerr-Schild r, and B -> 0;
  * Kerr in Kerr-Schild coordinates (a = 0.6): I -> 3 M^2 / (r - i a
    cos(theta))^6, the type-D value 3 Psi_2^2 with Psi_2 = -M / (r - i a
    cos(theta))^3 (r, theta Boyer-Lindquist), which fixes the sign of B.
"""
import numpy as np
import pytest

import exact
import oracle
from paper_1307_6488_gb300 import inputs

ORDERS = [(4, (12, 24, 48), 3.5, 1.5), (8, (12, 16, 20), 6.0, 2.0)]


def interior(a, g):
    return a[..., g:-g, g:-g, g:-g]


def rate(e, ns):
    return np.log(e[0] / e[-1]) / np.log(ns[-1] / ns[0])


@pytest.mark.parametrize("order", [4, 8])
def test_flat_space_exact_zero(order):
    g = order // 2 + 1
    u = inputs.flat_space(7, 6, 5, g)
    r = oracle.psi4(u, g, 0.1, order, (-0.3, -0.25, 0.05))
    for k in ("psi4", "inv", "E", "B"):
        assert np.max(np.abs(r[k])) == 0.0, k


def test_kasner_electric_part_closed_form():
    u0, _, p = exact.kasner(p_u=1.5, t0=1.3)
    g, n, t = 3, 4, 1.3
    u = np.broadcast_to(u0[:, None, None, None], (24, n + 2 * g, n + 2 * g, n + 2 * g)).copy()
    r = oracle.psi4(u, g, 0.1, 4, (0.3, 0.4, 0.5))
    E = np.zeros((3, 3))
    for (i, j) in exact.PAIRS:
        E[i, j] = E[j, i] = r["E"][exact.SYM[i][j], g, g, g]
    W = u0[inputs.IDX["W"]]
    gt = np.zeros((3, 3))
    for (i, j) in exact.PAIRS:
        gt[i, j] = gt[j, i] = u0[inputs.IDX["gt11"] + exact.SYM[i][j]]
    gamu = W * W * np.linalg.inv(gt)
    ev = np.sort(np.linalg.eigvals(gamu @ E).real)
    want = np.sort([(q - q * q) / t ** 2 for q in p])
    np.testing.assert_allclose(ev, want, rtol=0, atol=1e-13)
    assert np.max(np.abs(r["B"])) < 1e-14


def _sphere_errors(n, order, lo, ext, make, R_of, M=1.0, er_of=None):
    g = order // 2 + 1
    h = ext / n
    X, Y, Z = exact.box(n, n, n, g, lo, h)
    u = make(X, Y, Z, M)
    r = oracle.psi4(u, g, h, order, tuple(l + 0.5 * h for l in lo))
    R = R_of(X, Y, Z, M)
    e_inv = np.max(np.abs(interior(r["inv"] - 3 * M * M / R ** 6, g)))
    e_psi = np.max(np.abs(interior(r["psi4"], g)))
    e_B = np.max(np.abs(interior(r["B"], g)))
    e_rr = None
    if er_of is not None:
        er = er_of(X, Y, Z, M)
        Err = sum(r["E"][exact.SYM[i][j]] * er[i] * er[j] for i in range(3) for j in range(3))
        e_rr = np.max(np.abs(interior(Err + 2 * M / R ** 3, g)))
    return e_inv, e_psi, e_B, e_rr


def _iso_R(X, Y, Z, M):
    r = np.sqrt(X * X + Y * Y + Z * Z)
    return r * (1 + M / (2 * r)) ** 2


def _iso_er(X, Y, Z, M):
    r = np.sqrt(X * X + Y * Y + Z * Z)
    psi2 = (1 + M / (2 * r)) ** 2
    return [X / (r * psi2), Y / (r * psi2), Z / (r * psi2)]


@pytest.mark.parametrize("order,ns,lo_rate,ext", ORDERS)
def test_isotropic_schwarzschild(order, ns, lo_rate, ext):
    lo = (0.6, 0.9, 1.2)
    e = [_sphere_errors(n, order, lo, ext, exact.isotropic_schwarzschild, _iso_R, er_of=_iso_er) for n in ns]
    assert max(x[2] for x in e) == 0.0  # K_ij = 0: B vanishes identically
    for q in (0, 1, 3):
        errs = [x[q] for x in e]
        assert rate(errs, ns) > lo_rate, (q, errs)


def _ks_R(X, Y, Z, M):
    return np.sqrt(X * X + Y * Y + Z * Z)


@pytest.mark.parametrize("order,ns,lo_rate,ext", ORDERS)
def test_kerr_schild_schwarzschild(order, ns, lo_rate, ext):
    lo = (0.9, 1.3, 1.1)
    e = [_sphere_errors(n, order, lo, ext, exact.kerr_schild, _ks_R) for n in ns]
    for q in (0, 1, 2):
        errs = [x[q] for x in e]
        assert rate(errs, ns) > lo_rate, (q, errs)


@pytest.mark.parametrize("order,ns,lo_rate,ext", ORDERS)
def test_kerr_invariant(order, ns, lo_rate, ext):
    a, M, lo = 0.6, 1.0, (0.9, 1.3, 1.1)
    errs, sizes = [], []
    for n in ns:
        g = order // 2 + 1
        h = ext / n
        X, Y, Z = exact.box(n, n, n, g, lo, h)
        u = exact.kerr_schild(X, Y, Z, M, a)
        r = oracle.psi4(u, g, h, order, tuple(l + 0.5 * h for l in lo))
        rr = exact.ks_radius([X, Y, Z], a)
        want = 3 * M * M / (rr - 1j * a * Z / rr) ** 6
        errs.append(np.max(np.abs(interior(r["inv"] - want, g))))
        sizes.append(np.max(np.abs(interior(want.imag, g))))
        assert np.max(np.abs(interior(r["B"], g))) > 1e-2  # rotation: B does not vanish
    assert rate(errs, ns) > lo_rate, errs
    assert errs[-1] < 1e-3 * sizes[-1]  # Im I is resolved, with its sign


def _bl_closed_form(X, Y, Z, masses, centers):
    """Two-puncture Brill-Lindquist data (time symmetric, gamma = psi^4
    delta): E_ij = R_ij of the conformally flat metric, from the textbook
    conformal-transformation formula with harmonic psi,
      R_ij = -2 d_i d_j psi / psi + 6 d_i psi d_j psi / psi^2 - 2 delta_ij |d psi|^2 / psi^2,
    and Psi_4 in the triad theta-hat / psi^2, phi-hat / psi^2 (the flat
    spherical unit vectors rescaled to unit length in gamma):
      Psi_4 = [ (E(th, th) - E(ph, ph)) / 2 - i E(th, ph) ] / psi^4."""
    x = [X, Y, Z]
    psi = np.ones_like(X)
    dpsi = [np.zeros_like(X) for _ in range(3)]
    ddpsi = [[np.zeros_like(X) for _ in range(3)] for _ in range(3)]
    for m, c in zip(masses, centers):
        d = [x[i] - c[i] for i in range(3)]
        r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
        psi = psi + m / (2 * r)
        for i in range(3):
            dpsi[i] = dpsi[i] - m * d[i] / (2 * r ** 3)
            for j in range(3):
                ddpsi[i][j] = ddpsi[i][j] + m * (3 * d[i] * d[j] - (r * r if i == j else 0.0)) / (2 * r ** 5)
    g2 = sum(dpsi[i] ** 2 for i in range(3))
    E = [[-2 * ddpsi[i][j] / psi + 6 * dpsi[i] * dpsi[j] / psi ** 2 - (2 * g2 / psi ** 2 if i == j else 0.0)
          for j in range(3)] for i in range(3)]
    rho = np.sqrt(X * X + Y * Y)
    rr = np.sqrt(X * X + Y * Y + Z * Z)
    th = [X * Z / (rho * rr), Y * Z / (rho * rr), -rho / rr]
    ph = [-Y / rho, X / rho, np.zeros_like(X)]
    q = lambda a, b: sum(E[i][j] * a[i] * b[j] for i in range(3) for j in range(3))
    return (0.5 * (q(th, th) - q(ph, ph)) - 1j * q(th, ph)) / psi ** 4


@pytest.mark.parametrize("order,ns,lo_rate,ext", ORDERS)
def test_brill_lindquist_psi4_closed_form(order, ns, lo_rate, ext):
    masses, centers = (0.3, 0.2), ((-0.8, 0.2, 0.1), (0.7, -0.3, -0.2))
    lo = (0.5, 0.7, 0.6)
    errs, size = [], None
    for n in ns:
        g = order // 2 + 1
        h = ext / n
        X, Y, Z = exact.box(n, n, n, g, lo, h)
        u = inputs.flat_space(n, n, n, g)
        psi = np.ones_like(X)
        for m, c in zip(masses, centers):
            psi = psi + m / (2 * np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2))
        u[inputs.IDX["W"]] = psi ** -2
        u[inputs.IDX["alpha"]] = psi ** -2
        r = oracle.psi4(u, g, h, order, tuple(l + 0.5 * h for l in lo))
        want = _bl_closed_form(X, Y, Z, masses, centers)
        errs.append(np.max(np.abs(interior(r["psi4"] - want, g))))
        size = np.max(np.abs(interior(want, g)))
        assert np.max(np.abs(r["B"])) == 0.0
    assert rate(errs, ns) > lo_rate, errs
    assert errs[-1] < 1e-3 * size and size > 1e-3
