"""GPU parity of the third-order Runge-Kutta method of lines (Sec. 3.3,
Shu-Osher SSP-RK3) through the C ABI against the oracle: each stage against
its definition built from oracle right-hand sides, 10 periodic steps of the
24^3 gauge wave (1e-10 per tensor field), static-boundary steps at both
orders, and the FP32-RHS form within its stated bound."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

from gpu_common import (RHS_TOL, STEPS_TOL, gauge_wave_c1, grid_for, need_gpu, oracle_params, perturbed_bl,
                        rel_err_tensor)

pytestmark = pytest.mark.gpu

W0 = [0.0, 0.75, 1.0 / 3.0]
W1 = [1.0, 0.25, 2.0 / 3.0]


@pytest.mark.parametrize("order", [4, 8])
def test_rk3_stages_parity(order):
    torch = need_gpu()
    g = order // 2 + 1
    u = perturbed_bl(12, 10, 14, g, 0.1, seed=31)
    inputs.periodic_wrap(u, g)
    p = B.make_params(fd_order=order)
    op = oracle_params(p)
    grid = grid_for(u, g, 0.1)
    dt = 0.025
    y0 = B.upload(u, grid)
    work = B.alloc_work(grid, p)
    ys, ys_np = y0, u.copy()
    I = (slice(None),) + (slice(g, -g),) * 3
    for s in range(3):
        k = oracle.rhs(ys_np, g, 0.1, op, ko=True)
        want = W0[s] * u + W1[s] * (ys_np + dt * k)
        ynext = B.alloc_state(grid)
        B.rk3_stage(grid, p, B.FP64, s, dt, y0, ys, ynext, work)
        torch.cuda.synchronize()
        got = B.download(ynext, grid)
        err = rel_err_tensor(got - u, want - u, g)  # relative to the stage's change
        assert np.max(err) < RHS_TOL, (s, dict(zip(inputs.VARS, err)))
        ys_np = want.copy()
        ys_np[I] = got[I]
        inputs.periodic_wrap(ys_np, g)
        ys = B.upload(ys_np, grid)


def test_rk3_ten_steps_gauge_wave_24():
    torch = need_gpu()
    u, h = gauge_wave_c1()
    g = 3
    p = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    op = oracle_params(p)
    dt = 0.25 * h
    grid = grid_for(u, g, h)
    state = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=2)
    work = B.alloc_work(grid, p)
    want = u.copy()
    for _ in range(10):
        B.rk3_step(grid, p, B.FP64, dt, 0, None, state, bufs, work)
        want = oracle.rk3_step(want, g, h, dt, op, bc=0)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    err = rel_err_tensor(got, want, g)
    assert np.max(err) < STEPS_TOL, dict(zip(inputs.VARS, err))
    assert np.array_equal(got, oracle.fill_ghosts(got.copy(), g, 0))


@pytest.mark.parametrize("order", [4, 8])
def test_rk3_steps_static_boundary(order):
    torch = need_gpu()
    g = order // 2 + 1
    u = perturbed_bl(14, 12, 10, g, 0.2, seed=29, amp=3e-3)
    p = B.make_params(fd_order=order)
    op = oracle_params(p)
    grid = grid_for(u, g, 0.2)
    state = B.upload(u, grid)
    src = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=2)
    work = B.alloc_work(grid, p)
    want = u.copy()
    for _ in range(3):
        B.rk3_step(grid, p, B.FP64, 0.05, 1, src, state, bufs, work)
        want = oracle.rk3_step(want, g, 0.2, 0.05, op, bc=1, ghost_src=u)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    err = rel_err_tensor(got - u, want - u, g)
    assert np.max(err) < STEPS_TOL, dict(zip(inputs.VARS, err))


def test_rk3_fp32_rhs_within_bound():
    """FP32-RHS RK3, 3 steps on smooth perturbed data: within the FP32 form's
    stated bound (1e-3 per tensor field of the change) against the oracle."""
    torch = need_gpu()
    g = 5
    u = perturbed_bl(16, 14, 12, g, 0.25, seed=37, amp=3e-3)
    p = B.make_params(fd_order=8)
    op = oracle_params(p)
    grid = grid_for(u, g, 0.25)
    state = B.upload(u, grid)
    src = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=2)
    work = B.alloc_work(grid, p, B.FP32_RHS)
    want = u.copy()
    for _ in range(3):
        B.rk3_step(grid, p, B.FP32_RHS, 0.05, 1, src, state, bufs, work)
        want = oracle.rk3_step(want, g, 0.25, 0.05, op, bc=1, ghost_src=u)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    err = rel_err_tensor(got - u, want - u, g)
    assert np.max(err) < 1e-3, dict(zip(inputs.VARS, err))
