"""2:1 restriction (orders 2 and 4) and tricubic prolongation through the C ABI against the
oracle (non-cubic ragged grids, all 24 variables)."""
import numpy as np
import pytest

import oracle
from paper_1307_6488_gb300 import binding as B

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order", [2, 4])
def test_restrict_matches_oracle(order):
    torch = need_gpu()
    rng = np.random.default_rng(5)
    fg, cg = 3, 4
    f = rng.standard_normal((24, 2 * 5 + 2 * fg, 2 * 7 + 2 * fg, 2 * 6 + 2 * fg))
    gf = B.make_grid(12, 14, 10, ghost=fg, dx=0.1)
    gc = B.make_grid(6, 7, 5, ghost=cg, dx=0.2)
    df = B.upload(f, gf)
    dc = B.alloc_state(gc)
    B.restrict(gf, df, gc, dc, order=order)
    torch.cuda.synchronize()
    want = oracle.restrict(f, fg, cg, order=order)
    I = (slice(None),) + (slice(cg, -cg),) * 3
    np.testing.assert_allclose(B.download(dc, gc)[I], want[I], rtol=1e-13, atol=1e-14)


def test_prolong_matches_oracle():
    torch = need_gpu()
    rng = np.random.default_rng(6)
    cg, fg = 2, 4
    c = rng.standard_normal((24, 5 + 2 * cg, 7 + 2 * cg, 6 + 2 * cg))
    gc = B.make_grid(6, 7, 5, ghost=cg, dx=0.2)
    gf = B.make_grid(12, 14, 10, ghost=fg, dx=0.1)
    dc = B.upload(c, gc)
    df = B.alloc_state(gf)
    B.prolong(gc, dc, gf, df)
    torch.cuda.synchronize()
    want = oracle.prolong(c, cg, fg)
    I = (slice(None),) + (slice(fg, -fg),) * 3
    np.testing.assert_allclose(B.download(df, gf)[I], want[I], rtol=1e-12, atol=1e-13)


def test_restrict_rejects_bad_order():
    need_gpu()
    gf = B.make_grid(8, ghost=0, dx=0.1)
    gc = B.make_grid(4, ghost=2, dx=0.2)
    df, dc = B.alloc_state(gf), B.alloc_state(gc)
    with pytest.raises(B.BssnError):
        B.restrict(gf, df, gc, dc, order=4)  # order 4 reads one fine ghost
    with pytest.raises(B.BssnError):
        B.restrict(B.make_grid(8, ghost=1, dx=0.1), df, gc, dc, order=3)
