"""Batched uneven patches in one graph launch per RK4 step (plan API):
each patch must step exactly as the single-grid path steps it (same
per-point arithmetic; static ghosts), for every tile shape the autotuner may
pick, in both precisions; one patch is also checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

from gpu_common import RHS_TOL, STEPS_TOL, grid_for, interior, need_gpu, oracle_params, rel_err_tensor

pytestmark = pytest.mark.gpu

SIZES = [(16, 24, 16), (24, 16, 32), (9, 12, 10), (20, 20, 20), (12, 33, 8), (40, 8, 17)]


def patch_state(n, g, h, origin, seed):
    """Brill-Lindquist patch data (tricubic fill) plus a seeded smooth
    perturbation so every variable and term is active."""
    w = inputs.bl_conformal_tricubic(n, g, h, origin)
    u = inputs.empty_state(*n, g)
    u[inputs.IDX["W"]] = w
    u[inputs.IDX["alpha"]] = w
    for i in range(3):
        u[inputs.IDX["gt11"] + inputs.SYM[i][i]] = 1.0
    inputs.smooth_perturbation(u, g, 2e-3, seed, h)
    return u


def make_patches(order, nsizes=len(SIZES)):
    g = 4 if order == 4 else 5
    out = []
    for b, n in enumerate(SIZES[:nsizes]):
        h = 0.5 / 2 ** (b % 3)
        origin = (0.3 + 0.1 * b, -0.4 + 0.05 * b, 0.2 - 0.07 * b)
        out.append((n, g, h, patch_state(n, g, h, origin, seed=300 + b)))
    return out


def step_single(u, g, h, p, prec, dt):
    torch = need_gpu()
    grid = grid_for(u, g, h)
    s = B.upload(u, grid)
    src = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p, prec)
    B.rk4_step(grid, p, prec, dt, 1, src, s, bufs, work)
    torch.cuda.synchronize()
    return B.download(s, grid)


@pytest.mark.parametrize("order,prec", [(4, B.FP64), (8, B.FP64), (4, B.FP32_RHS), (8, B.FP32_RHS)])
@pytest.mark.parametrize("autotune", [0, 1])
def test_batch_step_matches_single_grid(order, prec, autotune):
    torch = need_gpu()
    patches = make_patches(order)
    p = B.make_params(fd_order=order)
    dt = 0.02
    blocks, keep = [], []
    for (n, g, h, u) in patches:
        grid = grid_for(u, g, h)
        st = B.upload(u, grid)
        src = B.upload(u, grid)
        keep.append((grid, st, src))
        blocks.append((grid, st, src))
    plan = B.plan_create(blocks, p, prec, autotune)
    try:
        pts, tiles, shapes = B.plan_info(plan, len(blocks))
        assert pts == sum(np.prod(n) for (n, _, _, _) in patches)
        assert np.all((shapes >= 0) & (shapes < 7))
        if prec == B.FP32_RHS:
            assert np.all(shapes == 6)  # the tiled kernel's fixed 8 x 4 x 4 tiles
        elif autotune == 0:
            assert np.all(shapes == 0)
        for step in range(2):
            B.batch_step(plan, dt)
        torch.cuda.synchronize()
        for (n, g, h, u), (grid, st, _) in zip(patches, keep):
            want = step_single(step_single(u, g, h, p, prec, dt), g, h, p, prec, dt)
            got = B.download(st, grid)
            if prec == B.FP32_RHS:
                # the same tiled kernel, tables and conversions as the single
                # grid: bit for bit
                np.testing.assert_array_equal(got, want)
                continue
            err = rel_err_tensor(got - u, want - u, g)
            assert np.max(err) < RHS_TOL, (n, dict(zip(inputs.VARS, err)))
    finally:
        B.plan_destroy(plan)


def test_batch_patch_vs_oracle():
    """One small patch of a batch of three against the CPU oracle (8th order,
    static ghosts, 2 steps)."""
    torch = need_gpu()
    patches = make_patches(8, nsizes=3)
    p = B.make_params(fd_order=8)
    dt = 0.02
    blocks = []
    for (n, g, h, u) in patches:
        grid = grid_for(u, g, h)
        blocks.append((grid, B.upload(u, grid), B.upload(u, grid)))
    plan = B.plan_create(blocks, p, B.FP64, 1)
    try:
        B.batch_step(plan, dt)
        B.batch_step(plan, dt)
        torch.cuda.synchronize()
        n, g, h, u = patches[2]
        want = u.copy()
        for _ in range(2):
            want = oracle.rk4_step(want, g, h, dt, oracle_params(p), bc=1, ghost_src=u)
        got = B.download(blocks[2][1], blocks[2][0])
        err = rel_err_tensor(got - u, want - u, g)
        assert np.max(err) < STEPS_TOL, dict(zip(inputs.VARS, err))
    finally:
        B.plan_destroy(plan)


def test_batch_dt_change_recaptures():
    """A new step size rebuilds the graph; stepping with dt then dt/2 equals
    the single-grid path doing the same."""
    torch = need_gpu()
    patches = make_patches(4, nsizes=2)
    p = B.make_params(fd_order=4)
    blocks = []
    for (n, g, h, u) in patches:
        grid = grid_for(u, g, h)
        blocks.append((grid, B.upload(u, grid), B.upload(u, grid)))
    plan = B.plan_create(blocks, p, B.FP64, 0)
    try:
        B.batch_step(plan, 0.02)
        B.batch_step(plan, 0.01)
        torch.cuda.synchronize()
        for (n, g, h, u), (grid, st, _) in zip(patches, blocks):
            want = step_single(step_single(u, g, h, p, B.FP64, 0.02), g, h, p, B.FP64, 0.01)
            err = rel_err_tensor(B.download(st, grid) - u, want - u, g)
            assert np.max(err) < RHS_TOL
    finally:
        B.plan_destroy(plan)
