"""Failure detection of the tensor-core kernels without a GPU fault: every
wait of the warp-specialised tcgen05 kernels gives up after a time limit,
records BSSN_ERR_TIMEOUT, and raises the CTA's abort flag so that the other
roles leave too, after which copies and MMAs in flight are waited for and
TMEM is freed. Here that path runs on purpose, with a 1 ms limit on a
barrier nothing arrives at; nothing traps, and the device stays usable for
the calls that follow in the same process."""
import time

import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B

from gpu_common import RHS_TOL, grid_for, need_gpu, oracle_params, perturbed_bl, rel_err

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_releases_everything():
    torch = need_gpu()
    t0 = time.perf_counter()
    st, flags = B.probe_wait_timeout(1_000_000)
    el = time.perf_counter() - t0
    assert st == B.ERR_TIMEOUT
    assert flags & 1, "TMEM was not freed"
    assert flags & 2, "the second role did not leave on the abort flag"
    # the second role's own limit is 2 s: it left on the flag, long before
    assert el < 1.5, el
    assert B.last_error() == B.OK


def test_device_usable_after_the_timeout():
    torch = need_gpu()
    st, _ = B.probe_wait_timeout(1_000_000)
    assert st == B.ERR_TIMEOUT
    # tensor cores: the MMA rate probe allocates TMEM and completes
    assert B.probe_mma_rate(32) > 0
    # and a right-hand side still matches the oracle
    g, h = 5, 0.12
    u = perturbed_bl(12, 10, 9, g, h, seed=77)
    p = B.make_params(fd_order=8)
    grid = grid_for(u, g, h)
    work = B.alloc_work(grid, p)
    out = B.alloc_state(grid)
    B.rhs(grid, p, B.FP64, B.upload(u, grid), out, work)
    torch.cuda.synchronize()
    want = oracle.rhs(u, g, h, oracle_params(p))
    assert np.max(rel_err(B.download(out, grid), want, g)) < RHS_TOL


def test_limits_are_checked():
    need_gpu()
    assert B.probe_wait_timeout(10)[0] == B.ERR_INVALID_ARG
    assert B.probe_wait_timeout(5_000_000_000)[0] == B.ERR_INVALID_ARG
