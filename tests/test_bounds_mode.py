"""The compile-time bounds-check mode (a substitute for a memory sanitizer):
the library builds with -DBSSN_BOUNDS_CHECK
into libbssn_check.so, reports the mode, and counts nothing until a kernel
runs. The GPU half (tests/test_gpu_bounds.py) runs parity cases on that
build and requires zero recorded violations."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_bounds_check_build_reports_its_mode():
    from paper_1307_6488_gb300 import build
    lib = build.build(bounds_check=True)
    assert lib.endswith("libbssn_check.so") and os.path.exists(lib)
    code = ("import sys; sys.path.insert(0, %r); from paper_1307_6488_gb300 import binding as B; "
            "print(B.LIB_PATH.endswith('libbssn_check.so'), B.bounds_check_enabled())" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, BSSN_BOUNDS_CHECK="1"),
                         capture_output=True, text=True, check=True).stdout.split()
    assert out == ["True", "True"]
    out = subprocess.run([sys.executable, "-c", code], env={k: v for k, v in os.environ.items()
                                                           if k != "BSSN_BOUNDS_CHECK"},
                         capture_output=True, text=True, check=True).stdout.split()
    assert out == ["False", "False"]
