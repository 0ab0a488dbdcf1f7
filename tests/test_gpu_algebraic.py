"""The algebraic constraints det(gt_ij) - 1 and gt^ij At_ij on the GPU
(bssn_algebraic_constraints, through the C ABI) against the oracle on the
same seeded inputs. Both are short products of stored values; the reduction
order differs, so the norms agree to a few ulps (bound 1e-12 relative)."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B
from paper_1307_6488_gb300 import inputs

from gpu_common import grid_for, need_gpu, perturbed_bl

pytestmark = pytest.mark.gpu


def _want(u, g):
    d, t = oracle.algebraic_constraints(u, g)
    return (np.array([np.sqrt(np.mean(d ** 2)), np.sqrt(np.mean(t ** 2))]),
            np.array([np.max(np.abs(d)), np.max(np.abs(t))]))


def _gpu(u, g, h, order=4):
    torch = need_gpu()
    p = B.make_params(fd_order=order)
    grid = grid_for(u, g, h)
    d = B.upload(u, grid)
    work = B.alloc_work(grid, p, B.FP64)
    out = B.algebraic_constraints(grid, p, d, work)
    torch.cuda.synchronize()
    return out


def test_flat_space_exact_zero():
    u = inputs.flat_space(9, 7, 6, 3)
    l2, mx, st = _gpu(u, 3, 0.1)
    assert st == B.OK and np.all(l2 == 0.0) and np.all(mx == 0.0)


@pytest.mark.parametrize("shape", [(19, 13, 11), (1, 1, 1), (130, 3, 2)])
def test_matches_oracle(shape):
    nx, ny, nz = shape
    g = 3
    u = perturbed_bl(nx, ny, nz, g, 0.12, seed=nx + ny, amp=5e-2)
    l2, mx, st = _gpu(u, g, 0.12)
    wl2, wmx = _want(u, g)
    assert st == B.OK
    assert np.all(wl2 > 1e-6)  # both really nonzero
    assert np.max(np.abs(l2 - wl2) / wl2) < 1e-12, (l2, wl2)
    assert np.max(np.abs(mx - wmx) / wmx) < 1e-12, (mx, wmx)


def test_nonfinite_reported():
    u = perturbed_bl(8, 8, 8, 3, 0.12)
    u[1, 6, 5, 4] = np.nan
    _, _, st = _gpu(u, 3, 0.12)
    assert st == B.ERR_NONFINITE


@pytest.mark.slow
def test_full_size_after_one_step():
    """The 128^3 Brill-Lindquist benchmark grid (det gt = 1 and At = 0
    exactly at t = 0) after one FP64 RK4 step: the drift the evolution leaves
    in both constraints, GPU against the oracle on the GPU's state. Both are
    at rounding level there (det gt - 1 ~ 1e-14, the trace a cancellation
    residue of At entries ~1e-4), so the two evaluation orders agree to a
    few ulps of the terms: 1e-15 absolute for det gt - 1, 1e-14 max|At| for
    the trace."""
    torch = need_gpu()
    g = 5
    u, h = inputs.brill_lindquist(128, g, lo=-8.0, hi=8.0)
    p = B.make_params(fd_order=8)
    grid = grid_for(u, g, h)
    src = B.upload(u, grid)
    state = src.clone()
    bufs = B.alloc_state(grid, n=3)
    work = B.alloc_work(grid, p, B.FP64)
    B.rk4_step(grid, p, B.FP64, 0.25 * h, 1, src, state, bufs, work)
    l2, mx, st = B.algebraic_constraints(grid, p, state, work)
    torch.cuda.synchronize()
    got = B.download(state, grid)
    wl2, wmx = _want(got, g)
    assert st == B.OK and np.all(wl2 > 0)
    tol = np.array([1e-15, 1e-14 * np.max(np.abs(got[8:14, g:-g, g:-g, g:-g]))])
    assert np.all(np.abs(l2 - wl2) <= 1e-12 * wl2 + tol), (l2, wl2, tol)
    assert np.all(np.abs(mx - wmx) <= 1e-12 * wmx + tol), (mx, wmx, tol)
