"""The oracle against its stored values (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): a regression pin that a
later change to the oracle's arithmetic must either keep or regenerate with a
stated reason. The physics pins of the same functions live in
test_oracle_physics.py."""
import os
import sys

import numpy as np
import pytest

import oracle

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


@pytest.mark.parametrize("case", sorted(make_golden.CASES))
def test_rhs_samples_reproduce(case):
    lin0, want = make_golden.load(case)
    g, lin, got = make_golden.compute(case)
    np.testing.assert_array_equal(lin, lin0)
    # per-variable relative to the variable's largest stored value (libm
    # differences between hosts stay far below this)
    scale = np.maximum(np.abs(want).max(axis=0), 1e-300)
    assert np.max(np.abs(got - want) / scale) < 1e-12


def test_golden_rhs_is_not_trivial():
    for case in make_golden.CASES:
        _, want = make_golden.load(case)
        assert want.shape == (make_golden.NPTS, 24)
        assert np.all(np.isfinite(want))
        # every variable's sampled right-hand side is non-zero somewhere (with
        # frozen shift, beta and B carry the dissipation term alone)
        assert (np.abs(want).max(axis=0) > 0).all()
