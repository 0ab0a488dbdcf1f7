"""GPU parity: the CUDA library through its C ABI against the FP64 oracle,
element by element, on seeded inputs (right-hand side of Sec. 1.1,
8th/4th-order stencils of Sec. 2.3/3.3, RK method of lines of Sec. 3.3).
Tolerances: 1e-12 per-variable relative for one right-hand side, 1e-10
after 10 RK4 steps (double precision)."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs
from paper_1307_6488_gb300.inputs import IDX, NVAR

from gpu_common import (RHS_TOL, STEPS_TOL, gauge_wave_c1, grid_for, interior, need_gpu, oracle_params,
                        perturbed_bl, rel_err, rel_err_tensor)

pytestmark = pytest.mark.gpu

GAUGES = [dict(lapse=0, shift=0, advect_gauge=1), dict(lapse=1, shift=0, advect_gauge=0),
          dict(lapse=2, shift=1, advect_gauge=1)]


def gpu_rhs(u, g, h, p, ko=False):
    torch = need_gpu()
    grid = grid_for(u, g, h)
    d = B.upload(u, grid)
    out = B.alloc_state(grid)
    work = B.alloc_work(grid, p)
    B.rhs(grid, p, B.FP64, d, out, work)
    if ko:
        B.ko_dissipation(grid, p, B.FP64, d, out)
    torch.cuda.synchronize()
    return B.download(out, grid)


@pytest.mark.parametrize("order", [4, 8])
def test_flat_space_exact_zero(order):
    torch = need_gpu()
    g = order // 2 + 1
    u = inputs.flat_space(13, 9, 7, g)
    p = B.make_params(fd_order=order)
    r = gpu_rhs(u, g, 0.1, p, ko=True)
    assert np.all(interior(r, g) == 0.0)
    grid = grid_for(u, g, 0.1)
    y0 = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    B.rk4_step(grid, p, B.FP64, 0.025, 0, None, y0, bufs, work)
    torch.cuda.synchronize()
    assert np.array_equal(B.download(y0, grid), u)


def test_rhs_parity_gauge_wave_24():
    """24^3 periodic gauge wave with 1e-10 noise, 4th order, 1+log,
    Gamma-driver (eta = 2): one right-hand side without and with KO."""
    u, h = gauge_wave_c1()
    g = 3
    p = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    for ko in (False, True):
        want = oracle.rhs(u, g, h, oracle_params(p), ko=ko)
        got = gpu_rhs(u, g, h, p, ko=ko)
        err = rel_err(got, want, g)
        assert np.max(err) < RHS_TOL, dict(zip(inputs.VARS, err))


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("gauge", GAUGES)
def test_rhs_parity_perturbed(order, gauge):
    """Ragged non-cubic grid, anisotropic spacing, every variable nonzero:
    the right-hand side without dissipation; with dissipation added too where
    every variable has a genuine right-hand side (1+log / harmonic with the
    Gamma-driver). With the frozen gauge, alpha, beta and B have dissipation
    only, which test_ko_parity measures against the operator norm."""
    g = order // 2 + 1
    nx, ny, nz = 19, 13, 11
    h = (0.11, 0.13, 0.12)
    u = perturbed_bl(nx, ny, nz, g, 0.12, seed=order + 3 * gauge["lapse"])
    p = B.make_params(fd_order=order, ko_eps=0.07, eta=1.7, shift_coeff=0.7, **gauge)
    for ko in ((False, True) if gauge["shift"] == 0 else (False,)):
        want = oracle.rhs(u, g, h, oracle_params(p), ko=ko)
        got = gpu_rhs(u, g, h, p, ko=ko)
        err = rel_err(got, want, g)
        assert np.max(err) < RHS_TOL, (ko, dict(zip(inputs.VARS, err)))


def ko_norm_err(got, want, u, g, eps, h):
    """Error of the dissipation term relative to the max-norm bound of the
    operator applied to the data, eps * sum_d (1/h_d) * max|u_v|: a
    (2r)-th difference of smooth data cancels to ~ (k h)^(2r) |u|, so its
    value relative to itself is only as accurate as ~4^r eps_mach/(k h)^(2r)
    in any summation order (the oracle's included)."""
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    scale = eps * (1 / hx + 1 / hy + 1 / hz) * np.max(np.abs(u.reshape(u.shape[0], -1)), axis=1)
    gi = interior(got, g).reshape(got.shape[0], -1)
    wi = interior(want, g).reshape(want.shape[0], -1)
    return np.max(np.abs(gi - wi), axis=1) / np.maximum(scale, 1e-300)


@pytest.mark.parametrize("order", [4, 8])
def test_ko_parity(order):
    g = order // 2 + 1
    u = perturbed_bl(10, 12, 9, g, 0.1, seed=5)
    p = B.make_params(fd_order=order, ko_eps=0.1)
    torch = need_gpu()
    grid = grid_for(u, g, 0.1)
    d = B.upload(u, grid)
    out = B.alloc_state(grid)
    B.ko_dissipation(grid, p, B.FP64, d, out)
    torch.cuda.synchronize()
    got = B.download(out, grid)
    want = oracle.ko(u, g, 0.1, oracle_params(p))
    err = ko_norm_err(got, want, u, g, 0.1, 0.1)
    assert np.max(err) < RHS_TOL, err
    # frozen gauge: the fused rhs + dissipation of alpha, beta, B is the dissipation alone
    pf = B.make_params(fd_order=order, ko_eps=0.1, lapse=2, shift=1)
    gotf = gpu_rhs(u, g, 0.1, pf, ko=True)
    wantf = oracle.rhs(u, g, 0.1, oracle_params(pf), ko=True)
    frozen = [IDX["alpha"]] + [IDX["beta1"] + i for i in range(3)] + [IDX["B1"] + i for i in range(3)]
    err = ko_norm_err(gotf[frozen], wantf[frozen], u[frozen], g, 0.1, 0.1)
    assert np.max(err) < RHS_TOL, err


@pytest.mark.parametrize("order", [4, 8])
def test_rk4_stages_parity(order):
    """Each of the four fused stages against the RK4 definition built from
    oracle right-hand sides: ynext = y0 + c_s dt k_s, acc = dt sum b_t k_t."""
    torch = need_gpu()
    g = order // 2 + 1
    u = perturbed_bl(12, 10, 14, g, 0.1, seed=11)
    inputs.periodic_wrap(u, g)
    p = B.make_params(fd_order=order)
    op = oracle_params(p)
    grid = grid_for(u, g, 0.1)
    dt = 0.025
    y0 = B.upload(u, grid)
    ys = y0
    acc = B.alloc_state(grid)
    work = B.alloc_work(grid, p)
    c = [0.5, 0.5, 1.0]
    b = [1 / 6, 1 / 3, 1 / 3, 1 / 6]
    ys_np = u.copy()
    acc_np = np.zeros_like(u)
    for s in range(4):
        k = oracle.rhs(ys_np, g, 0.1, op, ko=True)
        acc_np = acc_np + b[s] * dt * k
        want_next = u + (c[s] * dt * k if s < 3 else acc_np)
        ynext = B.alloc_state(grid)
        B.rk4_stage(grid, p, B.FP64, s, dt, y0, ys, acc, ynext, work)
        torch.cuda.synchronize()
        got = B.download(ynext, grid)
        scale = np.max(np.abs(interior(want_next - u, g)).reshape(NVAR, -1), axis=1) + 1e-300
        err = np.max(np.abs(interior(got - want_next, g)).reshape(NVAR, -1), axis=1) / scale
        assert np.max(err) < RHS_TOL, (s, dict(zip(inputs.VARS, err)))
        if s < 3:
            err_acc = rel_err(B.download(acc, grid), acc_np, g)
            assert np.max(err_acc) < RHS_TOL, (s, err_acc)
            ys_np = got.copy()
            oracle.fill_ghosts(ys_np, g, 0)
            ys = B.upload(ys_np, grid)


def test_ten_steps_gauge_wave_24():
    """24^3 gauge wave + noise, 4th order, KO 0.1, dt = 0.25 dx, 10 RK4 steps;
    error per tensor field (see rel_err_tensor)."""
    torch = need_gpu()
    u, h = gauge_wave_c1()
    g = 3
    p = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    op = oracle_params(p)
    dt = 0.25 * h
    grid = grid_for(u, g, h)
    state = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    want = u.copy()
    for _ in range(10):
        B.rk4_step(grid, p, B.FP64, dt, 0, None, state, bufs, work)
        want = oracle.rk4_step(want, g, h, dt, op, bc=0)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    err = rel_err_tensor(got, want, g)
    assert np.max(err) < STEPS_TOL, dict(zip(inputs.VARS, err))
    # ghosts refilled periodically
    assert np.array_equal(got, oracle.fill_ghosts(got.copy(), g, 0))


@pytest.mark.parametrize("order", [4, 8])
def test_steps_static_boundary(order):
    """Brill-Lindquist-like data, static ghosts, 3 steps, 1+log/Gamma-driver."""
    torch = need_gpu()
    g = order // 2 + 1
    u = perturbed_bl(14, 12, 10, g, 0.2, seed=23, amp=3e-3)
    p = B.make_params(fd_order=order)
    op = oracle_params(p)
    grid = grid_for(u, g, 0.2)
    state = B.upload(u, grid)
    src = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    want = u.copy()
    for _ in range(3):
        B.rk4_step(grid, p, B.FP64, 0.05, 1, src, state, bufs, work)
        want = oracle.rk4_step(want, g, 0.2, 0.05, op, bc=1, ghost_src=u)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    err = rel_err_tensor(got - u, want - u, g)  # relative to the change over the steps
    assert np.max(err) < STEPS_TOL, dict(zip(inputs.VARS, err))


@pytest.mark.parametrize("order", [4, 8])
def test_constraints_parity(order):
    torch = need_gpu()
    g = order // 2 + 1
    u = perturbed_bl(15, 11, 9, g, 0.15, seed=31)
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, 0.15)
    d = B.upload(u, grid)
    work = B.alloc_work(grid, p)
    ham = B.alloc_state(grid)
    mom = B.alloc_state(grid)
    gcon = B.alloc_state(grid)
    l2, mx, st = B.constraints(grid, p, d, work, ham=ham, mom=mom, gcon=gcon)
    assert st == B.OK
    wl2, wmx, wst, (wham, wmom, wg) = oracle.constraints(u, g, 0.15, order, fields=True)
    got = np.concatenate([B.download(ham, grid, 1), B.download(mom, grid, 3), B.download(gcon, grid, 3)])
    want = np.concatenate([wham[None], wmom, wg])
    err = rel_err(got, want, g)
    assert np.max(err) < RHS_TOL, err
    np.testing.assert_allclose(l2, wl2, rtol=1e-12)
    np.testing.assert_allclose(mx, wmx, rtol=1e-12)


@pytest.mark.parametrize("order", [4, 8])
def test_hamiltonian_alone_is_the_same_bits(order):
    """The Hamiltonian-only evaluation (the learned step's monitor) gives the
    full evaluation's H field and norms bit for bit, and its H against the
    oracle; a non-positive W at an interior point is still flagged."""
    torch = need_gpu()
    g = order // 2 + 1
    u = perturbed_bl(15, 11, 9, g, 0.15, seed=32)
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, 0.15)
    d = B.upload(u, grid)
    work = B.alloc_work(grid, p)
    ham = B.alloc_state(grid)
    ham1 = B.alloc_state(grid)
    l2, mx, st = B.constraints(grid, p, d, work, ham=ham)
    h2, hm, hst = B.hamiltonian(grid, p, d, work, ham=ham1)
    torch.cuda.synchronize()
    assert st == hst == B.OK
    assert h2 == l2[0] and hm == mx[0]
    gi = interior(B.download(ham, grid, 1), g)
    assert np.array_equal(interior(B.download(ham1, grid, 1), g), gi)
    wl2, wmx, wst, (wham, _, _) = oracle.constraints(u, g, 0.15, order, fields=True)
    assert rel_err(B.download(ham1, grid, 1), wham[None], g)[0] < RHS_TOL
    u[IDX["W"], g + 1, g + 5, g + 2] = -0.25
    assert B.hamiltonian(grid, p, B.upload(u, grid), work)[2] == B.ERR_NONFINITE


def test_constraints_nonfinite_status():
    torch = need_gpu()
    g = 3
    u = perturbed_bl(8, 8, 8, g, 0.15, seed=3)
    u[IDX["trK"], g + 2, g + 3, g + 4] = np.nan
    p = B.make_params(fd_order=4)
    grid = grid_for(u, g, 0.15)
    d = B.upload(u, grid)
    work = B.alloc_work(grid, p)
    l2, mx, st = B.constraints(grid, p, d, work)
    assert st == B.ERR_NONFINITE


def test_constraints_flag_nonpositive_conformal_factor():
    """A finite but non-positive W at one interior point is reported like a
    non-finite value; the same state with W > 0 there is not."""
    torch = need_gpu()
    g = 3
    u = perturbed_bl(8, 8, 8, g, 0.15, seed=4)
    p = B.make_params(fd_order=4)
    grid = grid_for(u, g, 0.15)
    work = B.alloc_work(grid, p)
    _, _, st = B.constraints(grid, p, B.upload(u, grid), work)
    assert st == B.OK
    u[IDX["W"], g + 1, g + 5, g + 2] = -0.25
    _, _, st = B.constraints(grid, p, B.upload(u, grid), work)
    assert st == B.ERR_NONFINITE


@pytest.mark.parametrize("mode", [0, 1])
def test_fill_ghosts_parity(mode):
    torch = need_gpu()
    g = 5
    rng = np.random.default_rng(2)
    u = rng.standard_normal((NVAR, 4 + 2 * g, 7 + 2 * g, 3 + 2 * g))  # n < g on some axes
    src = rng.standard_normal(u.shape)
    grid = grid_for(u, g, 1.0)
    d = B.upload(u, grid)
    s = B.upload(src, grid)
    B.fill_ghosts(grid, mode, s if mode == 1 else None, d)
    torch.cuda.synchronize()
    want = oracle.fill_ghosts(u.copy(), g, mode, src if mode == 1 else None)
    assert np.array_equal(B.download(d, grid), want)


def test_single_point_grid():
    """Degenerate 1x1x1 periodic grid: every stencil wraps onto one point."""
    torch = need_gpu()
    g = 3
    u = inputs.flat_space(1, 1, 1, g)
    inputs.add_noise(u, g, 1e-3, 99, periodic=True)
    oracle.fill_ghosts(u, g, 0)
    p = B.make_params(fd_order=4)
    want = oracle.rhs(u, g, 0.1, oracle_params(p), ko=True)
    got = gpu_rhs(u, g, 0.1, p, ko=True)
    np.testing.assert_allclose(interior(got, g), interior(want, g), rtol=1e-12, atol=1e-13)


@pytest.mark.slow
def test_full_size_128_sampled():
    """128^3 Brill-Lindquist (bare masses 0.5 at x = +-1.5, [-8, 8]^3),
    8th order, 5 ghosts, static boundary; plus a seeded 1e-3 perturbation so
    every term is active. One fused RK4 stage 0 in the launch configuration
    the benchmark times, checked at 4096 sampled points against the oracle."""
    torch = need_gpu()
    g, n = 5, 128
    u, h = inputs.brill_lindquist(n, g)
    inputs.smooth_perturbation(u, g, 1e-3, 4242, h)
    p = B.make_params(fd_order=8)
    grid = grid_for(u, g, h)
    y0 = B.upload(u, grid)
    acc = B.alloc_state(grid)
    ynext = B.alloc_state(grid)
    work = B.alloc_work(grid, p)
    dt = 0.25 * h
    B.rk4_stage(grid, p, B.FP64, 0, dt, y0, y0, acc, ynext, work)
    torch.cuda.synchronize()
    rng = np.random.default_rng(128)
    lin = np.unique(rng.integers(0, n ** 3, 4096))
    k = oracle.rhs_points(u, g, h, oracle_params(p), lin, ko=True)  # (npts, 24)
    got_acc = B.download(acc, grid)
    gi = interior(got_acc, g).reshape(NVAR, -1)[:, lin].T
    want = dt / 6 * k
    scale = np.max(np.abs(want), axis=0) + 1e-300
    err = np.max(np.abs(gi - want), axis=0) / scale
    assert np.max(err) < RHS_TOL, dict(zip(inputs.VARS, err))


def test_rk4_steps_capture_in_a_cuda_graph():
    """bssn_rk4_step launches only on the given stream and allocates
    nothing, so a sequence of steps can be captured in a CUDA graph; the
    replay gives the eager result bit for bit (24^3 gauge wave, periodic)."""
    torch = need_gpu()
    u, h = gauge_wave_c1()
    g = 3
    p = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    grid = grid_for(u, g, h)
    a = B.upload(u, grid)
    b = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    for _ in range(3):
        B.rk4_step(grid, p, B.FP64, 0.25 * h, 0, None, a, bufs, work)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=side):
        for _ in range(3):
            B.rk4_step(grid, p, B.FP64, 0.25 * h, 0, None, b, bufs, work)
    b.copy_(B.upload(u, grid))
    torch.cuda.synchronize()
    cg.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("order", [4, 8])
@pytest.mark.parametrize("axis", [0, 2])
def test_reflection_symmetry(order, axis):
    """The GPU right-hand side (with dissipation) of a state reflected along
    one axis is the reflection of its right-hand side, each component signed
    by its parity (the oracle's reflection pin, here on the GPU path, whose
    upwind stencil is mirrored through the address): to 1e-13 of each
    variable's largest value."""
    g = order // 2 + 1
    u = perturbed_bl(17, 12, 10, g, 0.12, seed=21 + axis, amp=3e-2)
    p = B.make_params(fd_order=order, eta=1.5)
    sign = np.ones(24)
    for i in range(3):
        for j in range(i, 3):
            s = (-1.0) ** ((i == axis) + (j == axis))
            sign[IDX["gt11"] + inputs.SYM[i][j]] = s
            sign[IDX["At11"] + inputs.SYM[i][j]] = s
    for base in ("Gt1", "beta1", "B1"):
        sign[IDX[base] + axis] = -1.0

    def reflect(s):
        return np.ascontiguousarray(np.flip(s, axis=3 - axis) * sign[:, None, None, None])

    r = gpu_rhs(u, g, 0.12, p, ko=True)
    r2 = gpu_rhs(reflect(u), g, 0.12, p, ko=True)
    want = reflect(r)
    scale = np.max(np.abs(interior(want, g)).reshape(24, -1), axis=1) + 1e-300
    err = np.max(np.abs(interior(r2 - want, g)).reshape(24, -1), axis=1) / scale
    assert np.max(err) < 1e-13, dict(zip(inputs.VARS, err))
    b = interior(u, g)[IDX["beta1"] + axis]
    assert b.min() < 0 < b.max()
