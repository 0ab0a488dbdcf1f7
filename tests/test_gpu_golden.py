"""The CUDA right-hand side (with Kreiss-Oliger dissipation, Sec. 3.3)
against the stored oracle values of tests/golden/: 24 sampled points of a
perturbed Brill-Lindquist block, 8th and 4th order, per-variable relative
tolerance 1e-12 (the stored values come from the oracle alone)."""
import os
import sys

import numpy as np
import pytest

from paper_1307_6488_gb300 import binding as B

from gpu_common import RHS_TOL, grid_for, need_gpu

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", sorted(make_golden.CASES))
def test_rhs_matches_golden(case):
    torch = need_gpu()
    kw = make_golden.CASES[case]
    g = kw["fd_order"] // 2 + 1
    u = make_golden.block(g)
    lin, want = make_golden.load(case)
    grid = grid_for(u, g, make_golden.H)
    p = B.make_params(**kw)
    d = B.upload(u, grid)
    out = B.alloc_state(grid)
    B.rhs(grid, p, B.FP64, d, out, B.alloc_work(grid, p))
    B.ko_dissipation(grid, p, B.FP64, d, out)
    torch.cuda.synchronize()
    got = B.download(out, grid)[:, g:-g, g:-g, g:-g].reshape(24, -1)[:, lin].T
    scale = np.abs(want).max(axis=0)
    err = np.abs(got - want).max(axis=0) / scale
    assert err.max() < RHS_TOL, err
