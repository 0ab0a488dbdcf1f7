"""bssn_rk4_stage_noalloc: the RK4 stage for callers that may not allocate
device memory (for example a plugin inside an application that owns the
device memory budget, or a loop that must not pay cudaMalloc's implicit
synchronisation). Its scratch is a static device array in the library, so it
must give the same results as bssn_rk4_stage with a caller-allocated work
buffer, call after call, and must refuse grids whose scratch would not fit.

This file is collected last on purpose: a failure here leaves every other
test already run."""
import numpy as np
import pytest

from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

import oracle

from gpu_common import RHS_TOL, grid_for, interior, need_gpu, oracle_params, perturbed_bl, rel_err_tensor

# the single-precision right-hand side against the FP64 oracle, per tensor
# field (the bound of the FP32-RHS tests)
FP32_RHS_TOL = 3e-4

pytestmark = pytest.mark.gpu


def _stage_both_ways(grid, p, prec, stage, dt, y0, ys, acc_in):
    """Run the stage with bssn_rk4_stage (caller work buffer) and with
    bssn_rk4_stage_noalloc from the same inputs; return both outputs."""
    torch = need_gpu()
    work = B.alloc_work(grid, p, prec)
    acc_ref = acc_in.clone()
    acc_new = acc_in.clone()
    out_ref = B.alloc_state(grid)
    out_new = B.alloc_state(grid)
    B.rk4_stage(grid, p, prec, stage, dt, y0, ys, acc_ref, out_ref, work)
    B.rk4_stage_noalloc(grid, p, prec, stage, dt, y0, ys, acc_new, out_new)
    torch.cuda.synchronize()
    return (B.download(out_ref, grid), B.download(acc_ref, grid)), (B.download(out_new, grid),
                                                                   B.download(acc_new, grid))


def _max_rel(got, want, g):
    gi = interior(got, g).reshape(got.shape[0], -1)
    wi = interior(want, g).reshape(want.shape[0], -1)
    return np.max(np.max(np.abs(gi - wi), axis=1) / np.maximum(np.max(np.abs(wi), axis=1), 1e-300))


@pytest.mark.parametrize("prec", [B.FP64, B.FP32_RHS])
def test_noalloc_matches_stage_on_two_calls_in_a_row(prec):
    torch = need_gpu()
    g = 5
    h = 0.12
    # two different inputs, two consecutive calls (stage 0, then stage 1 on the
    # first call's output), each against the work-buffer entry point
    u = perturbed_bl(18, 14, 12, g, h, seed=101)
    inputs.periodic_wrap(u, g)
    grid = grid_for(u, g, h)
    p = B.make_params(fd_order=8)
    dt = 0.25 * h
    y0 = B.upload(u, grid)
    acc0 = B.alloc_state(grid)
    (ref1, racc1), (new1, nacc1) = _stage_both_ways(grid, p, prec, 0, dt, y0, y0, acc0)
    assert _max_rel(new1, ref1, g) < RHS_TOL
    assert _max_rel(nacc1, racc1, g) < RHS_TOL
    # and directly against the oracle: after stage 0, acc = dt/6 k(y0)
    k = oracle.rhs(u, g, h, oracle_params(p), ko=True)
    want = dt / 6 * k
    if prec == B.FP64:
        assert _max_rel(nacc1, want, g) < RHS_TOL
    else:
        assert np.max(rel_err_tensor(nacc1, want, g)) < FP32_RHS_TOL
    ys_np = inputs.periodic_wrap(ref1.copy(), g)
    ys = B.upload(ys_np, grid)
    acc1 = B.upload(racc1, grid)
    (ref2, racc2), (new2, nacc2) = _stage_both_ways(grid, p, prec, 1, dt, y0, ys, acc1)
    assert _max_rel(new2, ref2, g) < RHS_TOL
    assert _max_rel(nacc2, racc2, g) < RHS_TOL


def test_noalloc_fourth_order_after_eighth():
    """A smaller 4th-order grid after the 8th-order calls: the shared scratch
    keeps the previous call's contents, which must not leak into results."""
    torch = need_gpu()
    g = 3
    u = perturbed_bl(11, 9, 13, g, 0.1, seed=202)
    inputs.periodic_wrap(u, g)
    grid = grid_for(u, g, 0.1)
    p = B.make_params(fd_order=4)
    y0 = B.upload(u, grid)
    acc = B.alloc_state(grid)
    for _ in range(2):
        (ref, racc), (new, nacc) = _stage_both_ways(grid, p, B.FP64, 0, 0.02, y0, y0, acc)
        assert _max_rel(new, ref, g) < RHS_TOL
        assert _max_rel(nacc, racc, g) < RHS_TOL


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = need_gpu()
    grid = B.make_grid(64, ghost=5, dx=0.1)
    p = B.make_params(fd_order=8)
    assert B.work_bytes(grid, p) > (64 << 20)
    # real states of this grid, so that even a call that got past the size
    # check would only touch live memory; the outputs must stay untouched
    y0, ys, acc, out = (B.alloc_state(grid) for _ in range(4))
    out.fill_(1.5)
    with pytest.raises(B.BssnError) as err:
        B.rk4_stage_noalloc(grid, p, B.FP64, 0, 0.01, y0, ys, acc, out)
    assert err.value.status == B.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((out == 1.5).all())
