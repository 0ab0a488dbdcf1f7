"""Refined hierarchy (Berger-Oliger, ratio 2 in space and time) and the
Sommerfeld outer boundary on the GPU, through the C ABI, against the
oracle's hierarchy stepping (oracle/amr.py) on the same seeded inputs.

Tolerances: one right-hand side of the radiative condition agrees to
rounding (1e-13 of its largest value); states after coarse steps are compared
per tensor field (gpu_common.rel_err_tensor) at 1e-10, the bound used for
states after several RK4 steps; the FP32-RHS form is bounded like
tests/test_gpu_fp32.py (1e-3 per tensor field after steps)."""
import numpy as np
import pytest

import oracle
from oracle import amr
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

from gpu_common import STEPS_TOL, need_gpu, oracle_params, rel_err_tensor

pytestmark = pytest.mark.gpu


def _bl_patch(o, n, g, h, xlo, seed):
    u = inputs.brill_lindquist_box(o, n, g, h, xlo, masses=(0.4, 0.3), centers=((-1.4, 0.1, 0.05), (1.6, -0.1, 0.1)))
    inputs.smooth_perturbation(u, g, 1e-3, seed, h)
    return u


def run_both(geo, ncells, xlo, h0, g, bc, p, dt0, steps, prec=B.FP64, data="bl"):
    """Evolve the same hierarchy with the GPU and the oracle; returns lists of
    (gpu, oracle) padded states per patch."""
    torch = need_gpu()
    us = []
    for b, (lev, o, n) in enumerate(geo):
        h = h0 / 2 ** lev
        if data == "bl":
            us.append(_bl_patch(o, n, g, h, xlo, seed=50 + b))
        else:
            us.append(inputs.gauge_wave_box(o, n, g, h, xlo, amplitude=0.05))
    grids = [B.make_grid(*n, ghost=g, dx=h0 / 2 ** lev) for (lev, o, n) in geo]
    dev = [B.upload(u, gr) for u, gr in zip(us, grids)]
    src = [B.upload(u, gr) for u, gr in zip(us, grids)]
    handle = B.amr_create([(lev, o, n, gr.var_stride, d, s if (bc == 1 and lev == 0) else None)
                           for (lev, o, n), gr, d, s in zip(geo, grids, dev, src)],
                          ncells, xlo, h0, g, bc, dt0, p, prec)
    try:
        for _ in range(steps):
            B.amr_step(handle)
        torch.cuda.synchronize()
        info = B.amr_info(handle)
    finally:
        B.amr_destroy(handle)
    got = [B.download(d, gr) for d, gr in zip(dev, grids)]
    pts = [amr.Patch(lev, o, n, u.copy(), ghost_src=u.copy()) for (lev, o, n), u in zip(geo, us)]
    H = amr.Hierarchy(pts, g, ncells, xlo, h0, bc, oracle_params(p), dt0)
    for _ in range(steps):
        H.step()
    assert info["updates_per_step"] == H.updates_per_step()
    return got, [q.state for q in H.P], info


def _check(got, want, g, tol):
    worst = 0.0
    for a, b in zip(got, want):
        worst = max(worst, float(np.max(rel_err_tensor(a, b, g))))
    assert worst < tol, worst
    return worst


def test_sommerfeld_rhs_matches_oracle():
    torch = need_gpu()
    g, n, h = 3, (14, 11, 9), (0.2, 0.25, 0.3)
    u = inputs.flat_space(*n, g)
    inputs.smooth_perturbation(u, g, 0.05, 11, 0.2)
    xyz0 = (3.1, -1.2, 0.7)
    p = B.make_params(fd_order=4, lapse=0)
    grid = B.make_grid(*n, ghost=g, dx=h[0], dy=h[1], dz=h[2])
    s = B.upload(u, grid)
    out = B.alloc_state(grid)
    B.sommerfeld_rhs(grid, p, xyz0, s, out)
    torch.cuda.synchronize()
    got = B.download(out, grid)
    want = amr.sommerfeld_rhs(u, h, xyz0, amr.radiative_speeds(oracle.Params(lapse=0)))
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
    # the asymptotic state gives exactly zero
    flat = B.upload(inputs.flat_space(*n, g), grid)
    B.sommerfeld_rhs(grid, p, xyz0, flat, out)
    torch.cuda.synchronize()
    assert np.all(B.download(out, grid) == 0.0)


def test_single_level_patches_periodic():
    """One level cut into three patches, periodic: sibling copies only."""
    g = 4
    p = B.make_params(fd_order=4, ko_eps=0.1, lapse=0, shift=0)
    geo = [(0, (0, 0, 0), (7, 12, 10)), (0, (7, 0, 0), (9, 12, 10)), (0, (16, 0, 0), (8, 12, 10))]
    got, want, info = run_both(geo, (24, 12, 10), (-0.5, 0, 0), 1.0 / 24, g, 0, p, 0.25 / 24, 3, data="gw")
    assert info["entries"]["prolong"] == 0 and info["entries"]["copy"] > 0
    _check(got, want, g, STEPS_TOL)


@pytest.mark.parametrize("prec", [B.FP64, B.FP32_RHS])
def test_two_levels_periodic_gauge_wave(prec):
    """Level 1 is the middle half in x, full in y and z (periodic images),
    cut into two patches; two coarse steps exercise both halves of the
    fine subcycle, prolongation from the parent's stage states and
    restriction."""
    g, N = 4, 16
    p = B.make_params(fd_order=4, ko_eps=0.1, lapse=1, shift=1)
    geo = [(0, (0, 0, 0), (N, 4, 4)), (1, (N // 2, 0, 0), (N // 2, 8, 8)), (1, (N, 0, 0), (N // 2, 8, 8))]
    got, want, info = run_both(geo, (N, 4, 4), (-0.5, 0.0, 0.0), 1.0 / N, g, 0, p, 0.25 / N, 2, prec=prec,
                               data="gw")
    assert info["entries"]["prolong"] > 0 and info["entries"]["restrict"] > 0 and info["levels"] == 2
    _check(got, want, g, STEPS_TOL if prec == B.FP64 else 1e-3)


@pytest.mark.parametrize("order,bc", [(8, 2), (4, 1), (4, 2)])
def test_three_levels_bl(order, bc):
    """The benchmark's hierarchy shape at small size: 8 patches on each of
    levels 0 and 1, a box around each puncture on level 2; radiative or
    static outer boundary; 1+log slicing and Gamma-driver shift."""
    g = 5 if order == 8 else 4
    ncells, xlo, h0, geo = inputs.bl_hierarchy(n0=16, nested=2, fine_half=4, split=2, extent=16.0)
    p = B.make_params(fd_order=order, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    got, want, info = run_both(geo, ncells, xlo, h0, g, bc, p, 0.25 * h0, 2)
    e = info["entries"]
    assert e["copy"] > 0 and e["prolong"] > 0 and e["restrict"] > 0
    assert (e["radiative"] > 0) == (bc == 2) and (e["static"] > 0) == (bc == 1)
    _check(got, want, g, STEPS_TOL)


def test_one_static_patch_equals_uniform_step():
    """A hierarchy of one level-0 patch with the static boundary is the
    uniform grid: bit for bit the result of bssn_rk4_step."""
    torch = need_gpu()
    g, n = 5, (14, 11, 9)
    h0 = 0.3
    xlo = (-2.0, -1.6, -1.3)
    u = _bl_patch((0, 0, 0), n, g, h0, xlo, seed=77)
    p = B.make_params(fd_order=8, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    grid = B.make_grid(*n, ghost=g, dx=h0)
    a = B.upload(u, grid)
    src = B.upload(u, grid)
    h = B.amr_create([(0, (0, 0, 0), n, grid.var_stride, a, src)], n, xlo, h0, g, 1, 0.25 * h0, p)
    try:
        for _ in range(3):
            B.amr_step(h)
    finally:
        B.amr_destroy(h)
    b = B.upload(u, grid)
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p)
    for _ in range(3):
        B.rk4_step(grid, p, B.FP64, 0.25 * h0, 1, src, b, bufs, work)
    torch.cuda.synchronize()
    assert np.array_equal(B.download(a, grid), B.download(b, grid))


def test_three_levels_bl_fp32_rhs():
    g = 5
    ncells, xlo, h0, geo = inputs.bl_hierarchy(n0=16, nested=2, fine_half=4, split=2, extent=16.0)
    p = B.make_params(fd_order=8, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    got, want, info = run_both(geo, ncells, xlo, h0, g, 2, p, 0.25 * h0, 2, prec=B.FP32_RHS)
    _check(got, want, g, 1e-3)


def test_flat_space_exact_full_benchmark_hierarchy():
    """The benchmark's own hierarchy (96^3 cells per level, 5 levels, 34
    patches, 8th order, radiative boundary): flat space stays bit-for-bit
    flat through a coarse step, in the launch configuration the benchmark
    times."""
    torch = need_gpu()
    g = 5
    ncells, xlo, h0, geo = inputs.bl_hierarchy()
    p = B.make_params(fd_order=8, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    grids = [B.make_grid(*n, ghost=g, dx=h0 / 2 ** lev) for (lev, o, n) in geo]
    flat = [inputs.flat_space(*n, g) for (lev, o, n) in geo]
    dev = [B.upload(u, gr) for u, gr in zip(flat, grids)]
    h = B.amr_create([(lev, o, n, gr.var_stride, d, None) for (lev, o, n), gr, d in zip(geo, grids, dev)],
                     ncells, xlo, h0, g, 2, 0.25 * h0, p)
    try:
        B.amr_step(h)
        torch.cuda.synchronize()
        info = B.amr_info(h)
    finally:
        B.amr_destroy(h)
    assert info["levels"] == 5 and info["updates_per_step"] == 96 ** 3 * 15 + 2 * 48 ** 3 * 16
    for d, gr, u in zip(dev, grids, flat):
        assert np.array_equal(B.download(d, gr), u)


def test_not_properly_nested_rejected():
    torch = need_gpu()
    g = 4
    p = B.make_params(fd_order=4)
    geo = [(0, (0, 0, 0), (16, 16, 16)), (1, (8, 8, 8), (16, 16, 16)), (2, (0, 32, 32), (8, 8, 8))]
    grids = [B.make_grid(*n, ghost=g, dx=1.0 / 2 ** lev) for (lev, o, n) in geo]
    dev = [B.upload(inputs.flat_space(*n, g), gr) for (lev, o, n), gr in zip(geo, grids)]
    with pytest.raises(B.BssnError) as ex:
        B.amr_create([(lev, o, n, gr.var_stride, d, None) for (lev, o, n), gr, d in zip(geo, grids, dev)],
                     (16, 16, 16), (-8.0,) * 3, 1.0, g, 2, 0.25, p)
    assert ex.value.status == B.ERR_INVALID_ARG
    torch.cuda.synchronize()


def test_regrid_matches_oracle():
    """Step a three-level hierarchy, regrid it with the finest boxes moved
    (level 1 kept, level 0 unchanged and its arrays reused), check the new
    states against the oracle's regrid, then step again and compare."""
    torch = need_gpu()
    g = 5
    ncells, xlo, h0, geo = inputs.bl_hierarchy(n0=16, nested=2, fine_half=4, split=2, extent=16.0)
    p = B.make_params(fd_order=8, ko_eps=0.1, lapse=0, shift=0, eta=2.0)
    dt0 = 0.25 * h0
    us = [_bl_patch(o, n, g, h0 / 2 ** lev, xlo, seed=90 + b) for b, (lev, o, n) in enumerate(geo)]
    grids = [B.make_grid(*n, ghost=g, dx=h0 / 2 ** lev) for (lev, o, n) in geo]
    dev = [B.upload(u, gr) for u, gr in zip(us, grids)]
    h = B.amr_create([(lev, o, n, gr.var_stride, d, None) for (lev, o, n), gr, d in zip(geo, grids, dev)],
                     ncells, xlo, h0, g, 2, dt0, p)
    pts = [amr.Patch(lev, o, n, u.copy()) for (lev, o, n), u in zip(geo, us)]
    H = amr.Hierarchy(pts, g, ncells, xlo, h0, 2, oracle_params(p), dt0)
    B.amr_step(h)
    H.step()
    # move the two finest boxes by (2, 2, -2) fine cells and (-2, 0, 2)
    moved = {(22, 28, 28): (24, 30, 26), (34, 28, 28): (32, 28, 30)}
    geo2 = [(lev, moved.get(tuple(o), tuple(o)) if lev == 2 else tuple(o), n) for (lev, o, n) in geo]
    grids2 = [B.make_grid(*n, ghost=g, dx=h0 / 2 ** lev) for (lev, o, n) in geo2]
    dev2 = [d if lev == 0 else B.alloc_state(gr) for (lev, o, n), gr, d in zip(geo2, grids2, dev)]
    try:
        h2 = B.amr_regrid(h, [(lev, o, n, gr.var_stride, d, None) for (lev, o, n), gr, d in zip(geo2, grids2, dev2)])
    finally:
        B.amr_destroy(h)
    try:
        H2 = H.regrid(geo2)
        got = [B.download(d, gr) for d, gr in zip(dev2, grids2)]
        for a, q in zip(got, H2.P):
            scale = max(1.0, float(np.max(np.abs(q.state))))
            assert np.max(np.abs(a - q.state)) < 1e-12 * scale
        B.amr_step(h2)
        torch.cuda.synchronize()
        H2.step()
        got = [B.download(d, gr) for d, gr in zip(dev2, grids2)]
        _check(got, [q.state for q in H2.P], g, STEPS_TOL)
    finally:
        B.amr_destroy(h2)
