"""Pins for the oracle's Berger-Oliger hierarchy stepping and Sommerfeld
outer boundary (not GPU).

The paper runs on Carpet's block-structured grids and plans ratio-2
adaptive refinement (Sec. 1.1, Sec. 4) without printing the algorithm; the
oracle follows Berger & Oliger with time-interpolated prolongation. Pins:
  * the RK4 continuous extension is exact on cubic solutions, and the fine
    ghost values are the stage inputs the fine RK4 makes when the solution
    is quadratic in time;
  * the Sommerfeld right-hand side is second-order accurate on an exact
    outgoing spherical wave and exactly zero on the asymptotic state;
  * one level cut into several patches evolves bit for bit like the single
    grid (sibling ghost copies, periodic and static boundaries);
  * prolonged ghosts are exact on parent stage states that are tricubic in
    space and come from a solution quadratic in time;
  * restriction is exact on tricubic fine data and touches only the coarse
    cells the fine interior covers;
  * flat space stays exactly flat through a three-level step with the
    radiative boundary;
  * a two-level evolution of the gauge wave converges to the exact solution;
  * regridding onto the same boxes changes nothing, and onto moved boxes it
    copies the cells the old boxes cover and prolongs the rest exactly on
    tricubic data.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import amr
from paper_1307_6488_gb300 import inputs


def _rk4_stage_states(g, t0, dt, y0=0.0):
    """RK4 on the scalar ODE y' = g(t): the stage inputs and result, as the
    parent keeps them (y0, Y2, Y3, Y4, y1), and the slopes."""
    f1 = g(t0)
    Y2 = y0 + dt / 2 * f1
    f2 = g(t0 + dt / 2)
    Y3 = y0 + dt / 2 * f2
    f3 = g(t0 + dt / 2)
    Y4 = y0 + dt * f3
    f4 = g(t0 + dt)
    y1 = y0 + dt / 6 * (f1 + 2 * f2 + 2 * f3 + f4)
    return (y0, Y2, Y3, Y4, y1)


def test_dense_output_exact_on_cubic_solutions():
    """For y' = g(t), g quadratic, the solution is cubic and the RK4
    continuous extension reproduces it and its derivatives exactly."""
    a, b, c = 0.7, -1.3, 2.1
    g = lambda t: a + b * t + c * t * t  # noqa: E731
    y = lambda t: a * t + b * t * t / 2 + c * t ** 3 / 3  # noqa: E731
    dt = 0.37
    S = _rk4_stage_states(g, 0.0, dt)
    D = [S[j] - S[0] for j in range(1, 5)]
    for chi in (0, 0.25, 0.5, 0.75, 1):
        cy, c1, c2, c3 = amr.dense_taylor(chi)
        t = chi * dt
        got = [sum(float(w) * d for w, d in zip(cc, D)) for cc in (cy, c1, c2, c3)]
        want = [y(t), dt * g(t), dt * dt * (b + 2 * c * t), dt ** 3 * 2 * c]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_fine_ghosts_are_the_fine_rk4_stage_inputs():
    """For y' = g(t), g linear, the ghost value at every fine stage input of
    both halves equals the stage input that RK4 with half the step makes
    from the exact solution, and the fine result equals the solution."""
    a, b = 0.4, -2.3
    g = lambda t: a + b * t  # noqa: E731
    y = lambda t: a * t + b * t * t / 2  # noqa: E731
    dt = 0.29
    S = _rk4_stage_states(g, 0.0, dt)
    D = [S[j] - S[0] for j in range(1, 5)]
    for m in (0, 1):
        tf = m * dt / 2
        fine = _rk4_stage_states(g, tf, dt / 2, y0=y(tf))
        want = list(fine[:4]) + [fine[4]]
        for s in range(5):
            d = amr.fine_ghost_coeffs(m, s)
            got = S[0] + sum(w * dd for w, dd in zip(d, D))
            assert abs(got - want[s]) < 1e-15, (m, s, got, want[s])
        assert abs(want[4] - y(tf + dt / 2)) < 1e-15


def _spherical_wave(h, v=1.0, t=0.3):
    """u = u_inf + F(r - v t)/r, F(s) = exp(-(s - 5)^2), on a box away from
    the origin; returns (u, xyz0, exact d_t u) for all 24 variables."""
    n = int(round(2.0 / h))
    x = 4.0 + (np.arange(n) + 0.5) * h
    y = -1.0 + (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(y, y, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    s = r - v * t
    F = np.exp(-(s - 5.0) ** 2)
    dF = -2.0 * (s - 5.0) * F
    uinf = amr._UINF
    u = np.stack([uinf[k] + (1.0 + 0.1 * k) * F / r for k in range(24)])
    dt = np.stack([-(1.0 + 0.1 * k) * v * dF / r for k in range(24)])
    return u, (x[0], y[0], y[0]), dt


def test_sommerfeld_outgoing_wave_second_order():
    errs = []
    for h in (0.1, 0.05, 0.025):
        u, xyz0, exact = _spherical_wave(h)
        got = amr.sommerfeld_rhs(u, h, xyz0, np.ones(24))
        errs.append(np.max(np.abs(got - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.3 for o in orders), (errs, orders)


def test_sommerfeld_speed_enters_linearly():
    u, xyz0, exact = _spherical_wave(0.025, v=math.sqrt(2.0))
    sp = np.full(24, math.sqrt(2.0))
    got = amr.sommerfeld_rhs(u, 0.025, xyz0, sp)
    assert np.max(np.abs(got - exact)) < 2e-3 * np.max(np.abs(exact))
    p = oracle.Params(lapse=0)
    assert amr.radiative_speeds(p)[17] == math.sqrt(2.0) and amr.radiative_speeds(p)[0] == 1.0


def test_sommerfeld_asymptotic_state_is_zero():
    u = inputs.flat_space(6, 5, 4, 3)
    out = amr.sommerfeld_rhs(u, (0.1, 0.2, 0.3), (3.0, -1.0, 2.0), np.full(24, 1.3))
    assert np.all(out == 0.0)


def _split_level0(u, g, n, cuts, bc):
    """Cut the single grid u into patches along x at the given cells."""
    pts = []
    edges = [0] + list(cuts) + [n[0]]
    for a, b in zip(edges[:-1], edges[1:]):
        sub = u[:, :, :, a:b + 2 * g].copy()
        pts.append(amr.Patch(0, (a, 0, 0), (b - a, n[1], n[2]), sub, ghost_src=sub.copy() if bc == 1 else None))
    return pts


@pytest.mark.parametrize("bc", [0, 1])
def test_single_level_patches_equal_single_grid(bc):
    g, n = 3, (20, 9, 7)
    p = oracle.Params(fd_order=4, ko_eps=0.1, lapse=0, shift=0)
    u, h = inputs.gauge_wave(n[0], g, amplitude=0.05, noise=0.0, ny=n[1], nz=n[2])
    inputs.smooth_perturbation(u, g, 1e-3, seed=5, h=h, periodic=(bc == 0))
    dt = 0.25 * h
    H = amr.Hierarchy(_split_level0(u, g, n, [6, 13], bc), g, n, (-0.5, 0, 0), h, bc, p, dt)
    ref = u.copy()
    for _ in range(2):
        H.step()
        ref = oracle.rk4_step(ref, g, h, dt, p, bc=bc, ghost_src=u if bc == 1 else None)
    for q in H.P:
        a = int(q.o[0])
        np.testing.assert_array_equal(q.state[:, g:-g, g:-g, g:-g], ref[:, g:-g, g:-g, g + a:g + a + int(q.n[0])])


def _poly(x, y, z):
    return ((1.0 + 0.3 * x - 0.2 * x ** 2 + 0.05 * x ** 3) * (0.7 + 0.1 * y - 0.04 * y ** 2 + 0.03 * y ** 3)
            * (1.1 - 0.2 * z + 0.06 * z ** 2 - 0.02 * z ** 3))


def _two_levels(g=4, bc=1, fine=((8, 8, 8), (16, 16, 16)), n0=16):
    p = oracle.Params(fd_order=4, ko_eps=0.1)
    xlo = (-2.0, -1.5, -1.0)
    h0 = 0.25
    u0 = inputs.flat_space(n0, n0, n0, g)
    pts = [amr.Patch(0, (0, 0, 0), (n0,) * 3, u0, ghost_src=u0.copy())]
    pts.append(amr.Patch(1, fine[0], fine[1], inputs.flat_space(*fine[1], g)))
    return amr.Hierarchy(pts, g, (n0,) * 3, xlo, h0, bc, p, 0.25 * h0), xlo, h0


def test_prolonged_ghosts_exact():
    """Parent stage states P(x) * (y0, Y2, Y3, Y4, y1) of RK4 on y' = g(t),
    g linear, P tricubic: every prolonged fine ghost equals P(x_fine) times
    the fine RK4 stage input (or result) of the same ODE."""
    H, xlo, h0 = _two_levels()
    g = H.g
    par = H.P[0]
    x, y, z = inputs.box_coords(par.o, par.n, g, h0, xlo)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    P = _poly(X, Y, Z)
    gt = lambda t: 0.3 - 1.1 * t  # noqa: E731
    yt = lambda t: 1.0 + 0.3 * t - 0.55 * t * t  # noqa: E731
    dt = 0.4
    S = _rk4_stage_states(gt, 0.0, dt, y0=1.0)
    par.stages = tuple(np.broadcast_to(sj * P, par.state.shape).copy() for sj in S)
    fine = H.P[1]
    pl = H.plans[1]
    assert not pl["copy"] and sum(int(ok.sum()) for ok, _, _ in pl["prolong"]) == len(pl["dst"][0])
    xf, yf, zf = inputs.box_coords(fine.o, fine.n, g, h0 / 2, xlo)
    Zf, Yf, Xf = np.meshgrid(zf, yf, xf, indexing="ij")
    gz, gy, gx = pl["dst"]
    Pf = _poly(Xf, Yf, Zf)[gz, gy, gx]
    for m in (0, 1):
        tf = m * dt / 2
        fs = _rk4_stage_states(gt, tf, dt / 2, y0=yt(tf))
        for s in range(5):
            fine.state[...] = 0.0
            H._pcache.clear()
            H._fill(1, [None, fine.state], m, s)
            np.testing.assert_allclose(fine.state[5, gz, gy, gx], fs[s] * Pf, rtol=0, atol=1e-13)


def test_restriction_exact_and_local():
    H, xlo, h0 = _two_levels()
    g = H.g
    fine = H.P[1]
    xf, yf, zf = inputs.box_coords(fine.o, fine.n, g, h0 / 2, xlo)
    Zf, Yf, Xf = np.meshgrid(zf, yf, xf, indexing="ij")
    fine.state[...] = _poly(Xf, Yf, Zf)
    par = H.P[0]
    par.state[...] = -7.0
    H._restrict(0)
    x, y, z = inputs.box_coords(par.o, par.n, g, h0, xlo)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    # fine interior cells [8, 24) cover coarse [4, 12); the 4-cell fine run
    # 2c-1 .. 2c+2 stays inside for coarse c = 5 .. 10
    cov = np.zeros(par.state.shape[1:], dtype=bool)
    cov[g + 5:g + 11, g + 5:g + 11, g + 5:g + 11] = True
    np.testing.assert_allclose(par.state[3][cov], _poly(X, Y, Z)[cov], rtol=0, atol=1e-13)
    assert np.all(par.state[3][~cov] == -7.0)


def test_flat_space_stays_flat_three_levels_radiative():
    g = 4
    p = oracle.Params(fd_order=4, ko_eps=0.1)
    n0 = 16
    pts = [amr.Patch(0, (0, 0, 0), (8, 16, 16), inputs.flat_space(8, 16, 16, g)),
           amr.Patch(0, (8, 0, 0), (8, 16, 16), inputs.flat_space(8, 16, 16, g)),
           amr.Patch(1, (8, 8, 8), (16, 16, 16), inputs.flat_space(16, 16, 16, g)),
           amr.Patch(2, (24, 24, 24), (8, 16, 16), inputs.flat_space(8, 16, 16, g)),
           amr.Patch(2, (32, 24, 24), (8, 16, 16), inputs.flat_space(8, 16, 16, g))]
    H = amr.Hierarchy(pts, g, (n0,) * 3, (-8.0,) * 3, 1.0, 2, p, 0.25)
    assert H.plans[3]["copy"] and H.plans[3]["prolong"]
    assert H.plans[0]["boundary"].any()
    before = [q.state.copy() for q in H.P]
    H.step()
    H.step()
    for q, b in zip(H.P, before):
        np.testing.assert_array_equal(q.state, b)


def test_not_properly_nested_is_rejected():
    with pytest.raises(ValueError):  # outside the level's domain
        _two_levels(fine=((-2, 8, 8), (16, 16, 16)))
    g = 4
    p = oracle.Params(fd_order=4)
    pts = [amr.Patch(0, (0, 0, 0), (16,) * 3, inputs.flat_space(16, 16, 16, g)),
           amr.Patch(1, (8, 8, 8), (16,) * 3, inputs.flat_space(16, 16, 16, g)),
           amr.Patch(2, (0, 32, 32), (8,) * 3, inputs.flat_space(8, 8, 8, g))]
    with pytest.raises(ValueError):  # level-2 ghosts beyond the level-1 patch
        amr.Hierarchy(pts, g, (16,) * 3, (-8.0,) * 3, 1.0, 2, p, 0.25)


def _gauge_wave_error(N, T=0.125):
    """Two-level periodic hierarchy: level 0 = N x 4 x 4 cells on
    [-0.5, 0.5) in x; level 1 = the middle half in x, full in y and z, cut
    into two patches. Harmonic slicing, frozen zero shift: the gauge wave is
    an exact solution. Returns the max error over all interior points."""
    g = 4
    p = oracle.Params(fd_order=4, ko_eps=0.1, lapse=1, shift=1)
    h0 = 1.0 / N
    xlo = (-0.5, 0.0, 0.0)
    A = 0.01
    geo = [(0, (0, 0, 0), (N, 4, 4)), (1, (N // 2, 0, 0), (N // 2, 8, 8)), (1, (N, 0, 0), (N // 2, 8, 8))]
    pts = [amr.Patch(l, o, n, inputs.gauge_wave_box(o, n, g, h0 / 2 ** l, xlo, amplitude=A)) for l, o, n in geo]
    dt = 0.25 * h0
    H = amr.Hierarchy(pts, g, (N, 4, 4), xlo, h0, 0, p, dt)
    steps = int(round(T / dt))
    for _ in range(steps):
        H.step()
    err = 0.0
    for (l, o, n), q in zip(geo, H.P):
        ex = inputs.gauge_wave_box(o, n, g, h0 / 2 ** l, xlo, amplitude=A, t=steps * dt)
        err = max(err, np.max(np.abs(q.state - ex)[:, g:-g, g:-g, g:-g]))
    return err


@pytest.mark.slow
def test_gauge_wave_two_levels_converges():
    e = [_gauge_wave_error(N) for N in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert e[0] < 1e-4, e
    assert min(orders) > 2.0, (e, orders)


def _geo_regrid(fine):
    return [(0, (0, 0, 0), (16, 16, 16)), (1, fine[0], fine[1])]


def test_regrid_same_boxes_is_identity():
    H, xlo, h0 = _two_levels()
    rng = np.random.default_rng(0)
    for q in H.P:
        q.state[...] = rng.standard_normal(q.state.shape)
    R = H.regrid(_geo_regrid(((8, 8, 8), (16, 16, 16))))
    for a, b in zip(H.P, R.P):
        # the interiors and every ghost the old patch holds are copied
        np.testing.assert_array_equal(a.state[:, 4:-4, 4:-4, 4:-4], b.state[:, 4:-4, 4:-4, 4:-4])
    np.testing.assert_array_equal(H.P[0].state, R.P[0].state)


def test_regrid_moved_box_copies_and_prolongs_exactly():
    """The fine box moves by (4, 2, 0) fine cells: cells still inside the old
    box are copied (bit for bit), the others are the tricubic prolongation of
    the parent, exact on tricubic data."""
    H, xlo, h0 = _two_levels()
    g = H.g
    par = H.P[0]
    x, y, z = inputs.box_coords(par.o, par.n, g, h0, xlo)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    par.state[...] = _poly(X, Y, Z)
    fine = H.P[1]
    fine.state[...] = 3.25  # distinguishable from the polynomial
    R = H.regrid(_geo_regrid(((12, 10, 8), (16, 16, 16))))
    q = R.P[1]
    xf, yf, zf = inputs.box_coords(q.o, q.n, g, h0 / 2, xlo)
    Zf, Yf, Xf = np.meshgrid(zf, yf, xf, indexing="ij")
    G = [np.arange(-g, 16 + g) + q.o[a] for a in range(3)]
    inside = ((G[0] >= 8) & (G[0] < 24))[None, None, :] & ((G[1] >= 8) & (G[1] < 24))[None, :, None] & \
        ((G[2] >= 8) & (G[2] < 24))[:, None, None]
    assert np.all(q.state[3][inside] == 3.25)
    np.testing.assert_allclose(q.state[3][~inside], _poly(Xf, Yf, Zf)[~inside], rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        H.regrid([(0, (0, 0, 0), (8, 16, 16))])
