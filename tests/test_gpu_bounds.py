"""Parity cases of the single-grid stencils (FP64 and FP32-RHS), the
constraints, Psi_4, batched patches, the refined hierarchy and the CFD
kernels, run on the bounds-check build of the library (libbssn_check.so):
every test must still pass and no kernel may record an access outside its
arrays (the conftest checks the device counters after each test)."""
import os
import subprocess
import sys

import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    "tests/test_gpu_parity.py",
    "tests/test_gpu_fp32.py::test_fp32_rhs_vs_oracle",
    "tests/test_gpu_fp32.py::test_fp32_whole_step_equals_its_stages",
    "tests/test_gpu_psi4.py",
    "tests/test_gpu_batch.py::test_batch_patch_vs_oracle",
    "tests/test_gpu_amr.py::test_two_levels_periodic_gauge_wave",
    "tests/test_gpu_amr.py::test_three_levels_bl",
    "tests/test_gpu_amr.py::test_regrid_matches_oracle",
    "tests/test_gpu_cfd.py::test_kernels_match_oracle",
    "tests/test_gpu_cfd.py::test_mass_iteration_equals_two_half_sweeps",
]


def test_parity_cases_on_the_bounds_check_build():
    need_gpu()
    from paper_1307_6488_gb300 import build
    build.build(bounds_check=True)
    env = dict(os.environ, BSSN_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider", *CASES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "error" not in r.stdout.lower().split("passed")[-1], tail
